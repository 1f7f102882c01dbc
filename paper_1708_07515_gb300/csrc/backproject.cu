// Cone-beam backprojection for FDK-OD (Sec. 2.2) and plain FDK (Sec. 2.1).
//
// One CTA of 16 x 16 threads owns a 16 x 16 column tile of one square and
// kZT consecutive slices; each thread owns one (x, y) column and kZT voxels
// along z in registers.  For every chunk of up to 8 views the CTA
//   1. finds, per view, the detector window its voxels can touch: the
//      column coordinate (Eq. 1 in square-local form) and the row
//      coordinate z/U + (Nv-1)/2 are monotone in x, y and z, so the tile's
//      corners bound them;
//   2. stages each window (rows x columns, zero outside the detector) from
//      global memory into shared memory with coalesced row loads;
//   3. accumulates U^-2 times the bilinear sample for each of its voxels.
// The gather is a sum over views of interpolated samples, not a dense
// contraction, so it runs on the FP32 pipes and the shared-memory path.
//
// Two sources share the kernel:
//   direct (D = 1 and the plain FDK baseline): Q_k itself, cropped per
//     (square, view) at crop = floor(phi + w0); column offset frac - w0;
//   decomposed (D > 1): the square's decimated data S'_q[j][v][t] at the
//     views beta_{jD}; column t = a - a_c - w0 (the second shift of
//     Sec. 2.1 folded into the addressing, as Sec. 2.2 says FDK-OD
//     interpolates once).
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <math.h>

#include <algorithm>
#include <utility>
#include <vector>

#include "fdkod_internal.cuh"
#include "tma.cuh"

namespace fdkod {
namespace {

constexpr int kThreads = kTile * kTile;
constexpr int kWarps = kThreads / 32;

struct BpParams {
    const void *src;
    float *vol;
    const GeomEntry *geo;
    const int32_t *crop;
    const int32_t *w0;
    int *status;
    long long sq_stride, view_stride, row_stride;  // source layout (elements)
    int src_cols, src_rows;
    int row0;                // detector row held in the source's row 0
    int zoff, nz;            // slices zoff .. zoff + nz - 1, written to vol[z - zoff]
    int N, P, Nv, m, tps;    // tps: tiles per square side
    int nviews, vstep;       // views summed; table view index = j * vstep
    int Wd, Rw, J;           // staging window and views per chunk
    float scale;             // pi / nviews
};

__device__ __forceinline__ float ld_s(const float *p) { return __ldg(p); }
__device__ __forceinline__ float ld_s(const __nv_bfloat16 *p) { return __bfloat162float(__ldg(p)); }
__device__ __forceinline__ float ld_s(const __half *p) { return __half2float(__ldg(p)); }

__device__ __forceinline__ void square_range(int q, int m, int N, int &i0, int &i1) {
    i0 = (int)(((long long)q * N + m - 1) / m);
    i1 = (int)((((long long)q + 1) * N + m - 1) / m) - 1;
}

template <typename TS, bool DIRECT>
__global__ void __launch_bounds__(kThreads)
bp_generic_kernel(BpParams a) {
    extern __shared__ float win[];
    __shared__ float s_cb[kViewsPerChunk], s_sb[kViewsPerChunk], s_r[kViewsPerChunk], s_al[kViewsPerChunk],
        s_ga[kViewsPerChunk], s_g[kViewsPerChunk], s_toff[kViewsPerChunk], s_vrel[kViewsPerChunk];
    __shared__ int s_vlo[kViewsPerChunk], s_col0[kViewsPerChunk];
    __shared__ long long s_off[kViewsPerChunk];

    const int tiles = a.tps * a.tps;
    const int q = blockIdx.x / tiles;
    const int tt = blockIdx.x - q * tiles;
    const int qy = q / a.m, qx = q - qy * a.m;
    int ix0, ix1, iy0, iy1;
    square_range(qx, a.m, a.N, ix0, ix1);
    square_range(qy, a.m, a.N, iy0, iy1);
    const int x0 = ix0 + (tt % a.tps) * kTile;
    const int y0 = iy0 + (tt / a.tps) * kTile;
    if (x0 > ix1 || y0 > iy1) return;  // ragged square: empty tile (uniform per CTA)
    const int xe = min(x0 + kTile - 1, ix1), ye = min(y0 + kTile - 1, iy1);
    const int z0 = a.zoff + blockIdx.y * kZT;
    const int z1 = min(z0 + kZT - 1, a.zoff + a.nz - 1);

    const float half_n = 0.5f * (float)(a.N - 1);
    const float xc = 0.5f * ((float)ix0 + (float)ix1) - half_n;  // square centre (exact half-integers)
    const float yc = 0.5f * ((float)iy0 + (float)iy1) - half_n;
    const float zc = 0.5f * ((float)z0 + (float)z1) - half_n;     // slab centre
    const double vcd = 0.5 * (double)(a.Nv - 1);

    const int lx = threadIdx.x % kTile, ly = threadIdx.x / kTile;
    const int x = x0 + lx, y = y0 + ly;
    const bool active = x <= xe && y <= ye;
    const float dx = (float)x - half_n - xc, dy = (float)y - half_n - yc;
    const float dz0 = (float)z0 - half_n - zc;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int WS = a.Wd + 1;
    const int32_t w0q = a.w0[q];

    float acc[kZT];
#pragma unroll
    for (int i = 0; i < kZT; ++i) acc[i] = 0.f;

    for (int jb = 0; jb < a.nviews; jb += a.J) {
        const int nj = min(a.J, a.nviews - jb);
        // 1. per-view window, one warp per view, lanes 0..7 take the corners
        if (warp < nj) {
            const int j = jb + warp;
            const int k = j * a.vstep;
            const size_t o = (size_t)q * a.P + k;
            const GeomEntry ge = a.geo[o];
            const float gf = ge.g_hi;
            const float toff = DIRECT ? ge.frac - (float)w0q : -(float)w0q;
            const int c = lane & 7;
            const float cx = (float)((c & 1) ? xe : x0) - half_n - xc;
            const float cy = (float)((c & 2) ? ye : y0) - half_n - yc;
            const float cz = (float)((c & 4) ? z1 : z0) - half_n - zc;
            const float dd = fmaf(ge.cb, cx, ge.sb * cy);
            const float invU = gf / fmaf(ge.r, dd, 1.0f);
            const float t = fmaf(invU, fmaf(ge.alpha, cx, ge.gamma * cy), toff);
            const float zq = zc * ge.r * dd;
            const double vcen = fma((double)zc, (double)ge.g_hi + (double)ge.g_lo, vcd);
            const double v = vcen + (double)(invU * (cz - zq));
            float tmin = t, tmax = t;
            double vmin = v, vmax = v;
#pragma unroll
            for (int off = 4; off > 0; off >>= 1) {
                tmin = fminf(tmin, __shfl_xor_sync(0xffffffffu, tmin, off));
                tmax = fmaxf(tmax, __shfl_xor_sync(0xffffffffu, tmax, off));
                vmin = fmin(vmin, __shfl_xor_sync(0xffffffffu, vmin, off));
                vmax = fmax(vmax, __shfl_xor_sync(0xffffffffu, vmax, off));
            }
            if (lane == 0) {
                const int tlo = (int)floorf(tmin) - 1;
                const int vlo = (int)floor(vmin) - 1;
                if ((int)floorf(tmax) + 2 - tlo > a.Wd - 1 || (int)floor(vmax) + 2 - vlo > a.Rw - 1)
                    atomicOr(a.status, 1);
                s_cb[warp] = ge.cb;
                s_sb[warp] = ge.sb;
                s_r[warp] = ge.r;
                s_al[warp] = ge.alpha;
                s_ga[warp] = ge.gamma;
                s_g[warp] = gf;
                s_toff[warp] = toff - (float)tlo;
                s_vrel[warp] = (float)(vcen - (double)vlo);
                s_vlo[warp] = vlo;
                if (DIRECT) {
                    const int col0 = a.crop[o] + tlo;
                    s_col0[warp] = col0;
                    s_off[warp] = (long long)k * a.view_stride + col0;
                } else {
                    s_col0[warp] = tlo;
                    s_off[warp] = (long long)q * a.sq_stride + (long long)j * a.view_stride + tlo;
                }
            }
        }
        __syncthreads();
        // 2. stage the windows: one warp per (view, row), lanes along columns
        const TS *src = (const TS *)a.src;
        for (int rid = warp; rid < nj * a.Rw; rid += kWarps) {
            const int w = rid / a.Rw;
            const int r = rid - w * a.Rw;
            const int v = s_vlo[w] + r - a.row0;  // row of the source
            const bool rok = v >= 0 && v < a.src_rows;
            const TS *row = src + s_off[w] + (long long)v * a.row_stride;
            float *dst = win + (size_t)rid * WS;
            const int col0 = s_col0[w];
            for (int c = lane; c < a.Wd; c += 32) {
                const int col = col0 + c;
                dst[c] = (rok && col >= 0 && col < a.src_cols) ? ld_s(row + c) : 0.f;
            }
        }
        __syncthreads();
        // 3. accumulate
        if (active) {
            for (int w = 0; w < nj; ++w) {
                const float dd = fmaf(s_cb[w], dx, s_sb[w] * dy);
                const float invU = s_g[w] / fmaf(s_r[w], dd, 1.0f);
                const float t = fmaf(invU, fmaf(s_al[w], dx, s_ga[w] * dy), s_toff[w]);
                const float tf = floorf(t);
                const float ft = t - tf;
                const int it = min(max((int)tf, 0), a.Wd - 2);
                const float wgt = invU * invU;
                const float zq = zc * s_r[w] * dd;
                const float vb = fmaf(-invU, zq, s_vrel[w]);
                const float *wp = win + (size_t)w * a.Rw * WS + it;
#pragma unroll
                for (int i = 0; i < kZT; ++i) {
                    const float v = fmaf(invU, dz0 + (float)i, vb);
                    const float vf = floorf(v);
                    const float fv = v - vf;
                    const int iv = min(max((int)vf, 0), a.Rw - 2);
                    const float *p = wp + iv * WS;
                    const float s00 = p[0], s01 = p[1], s10 = p[WS], s11 = p[WS + 1];
                    const float c0 = fmaf(ft, s01 - s00, s00);
                    const float c1 = fmaf(ft, s11 - s10, s10);
                    acc[i] = fmaf(wgt, fmaf(fv, c1 - c0, c0), acc[i]);
                }
            }
        }
        __syncthreads();
    }
    if (active) {
#pragma unroll
        for (int i = 0; i < kZT; ++i)
            if (z0 + i <= z1) a.vol[((size_t)(z0 + i - a.zoff) * a.N + y) * a.N + x] = acc[i] * a.scale;
    }
}

// Unstaged form for windows too large to stage in shared memory (a source
// close to the volume magnifies a tile's footprint on the detector): the
// same tiling and arithmetic as bp_generic_kernel, every sample read from the
// source in global memory (zero outside it).  Row coordinates stay relative
// to an integer base row per view, as in the staged kernels.
template <typename TS, bool DIRECT>
__global__ void __launch_bounds__(kThreads)
bp_global_kernel(BpParams a) {
    const int tiles = a.tps * a.tps;
    const int q = blockIdx.x / tiles;
    const int tt = blockIdx.x - q * tiles;
    const int qy = q / a.m, qx = q - qy * a.m;
    int ix0, ix1, iy0, iy1;
    square_range(qx, a.m, a.N, ix0, ix1);
    square_range(qy, a.m, a.N, iy0, iy1);
    const int x0 = ix0 + (tt % a.tps) * kTile;
    const int y0 = iy0 + (tt / a.tps) * kTile;
    if (x0 > ix1 || y0 > iy1) return;
    const int xe = min(x0 + kTile - 1, ix1), ye = min(y0 + kTile - 1, iy1);
    const int z0 = a.zoff + blockIdx.y * kZT;
    const int z1 = min(z0 + kZT - 1, a.zoff + a.nz - 1);
    const float half_n = 0.5f * (float)(a.N - 1);
    const float xc = 0.5f * ((float)ix0 + (float)ix1) - half_n;
    const float yc = 0.5f * ((float)iy0 + (float)iy1) - half_n;
    const float zc = 0.5f * ((float)z0 + (float)z1) - half_n;
    const double vcd = 0.5 * (double)(a.Nv - 1);
    const int lx = threadIdx.x % kTile, ly = threadIdx.x / kTile;
    const int x = x0 + lx, y = y0 + ly;
    if (x > xe || y > ye) return;  // no block barrier below
    const float dx = (float)x - half_n - xc, dy = (float)y - half_n - yc;
    const float dz0 = (float)z0 - half_n - zc;
    const int32_t w0q = a.w0[q];
    const TS *src = (const TS *)a.src;
    auto at = [&](long long off, int r, int c) -> float {  // sample (row r of the detector, column c of the source)
        const int rr = r - a.row0;
        return (rr >= 0 && rr < a.src_rows && c >= 0 && c < a.src_cols) ? ld_s(src + off + (long long)rr * a.row_stride + c)
                                                                         : 0.f;
    };
    float acc[kZT];
#pragma unroll
    for (int i = 0; i < kZT; ++i) acc[i] = 0.f;
    for (int j = 0; j < a.nviews; ++j) {
        const int k = j * a.vstep;
        const size_t o = (size_t)q * a.P + k;
        const GeomEntry ge = a.geo[o];
        const float toff = DIRECT ? ge.frac - (float)w0q : -(float)w0q;
        const float dd = fmaf(ge.cb, dx, ge.sb * dy);
        const float invU = ge.g_hi / fmaf(ge.r, dd, 1.0f);
        const float t = fmaf(invU, fmaf(ge.alpha, dx, ge.gamma * dy), toff);
        const float tf = floorf(t);
        const float ft = t - tf;
        const int col = (DIRECT ? a.crop[o] : 0) + (int)tf;
        const long long off = DIRECT ? (long long)k * a.view_stride : (long long)q * a.sq_stride + (long long)j * a.view_stride;
        const float wgt = invU * invU;
        const double vcen = fma((double)zc, (double)ge.g_hi + (double)ge.g_lo, vcd);
        const int vbase = (int)floor(vcen);
        const float zq = zc * ge.r * dd;
        const float vb = fmaf(-invU, zq, (float)(vcen - (double)vbase));
#pragma unroll
        for (int i = 0; i < kZT; ++i) {
            const float v = fmaf(invU, dz0 + (float)i, vb);
            const float vf = floorf(v);
            const float fv = v - vf;
            const int r = vbase + (int)vf;
            const float s00 = at(off, r, col), s01 = at(off, r, col + 1);
            const float s10 = at(off, r + 1, col), s11 = at(off, r + 1, col + 1);
            const float c0 = fmaf(ft, s01 - s00, s00);
            const float c1 = fmaf(ft, s11 - s10, s10);
            acc[i] = fmaf(wgt, fmaf(fv, c1 - c0, c0), acc[i]);
        }
    }
#pragma unroll
    for (int i = 0; i < kZT; ++i)
        if (z0 + i <= z1) a.vol[((size_t)(z0 + i - a.zoff) * a.N + y) * a.N + x] = acc[i] * a.scale;
}

template <typename TS, bool DIRECT>
cudaError_t launch_t(BpParams prm, int nsq, cudaStream_t st) {
    if (prm.J < 1) {  // one view's window does not fit shared memory: sample from global memory
        dim3 grid((unsigned)(nsq * prm.tps * prm.tps), (unsigned)((prm.nz + kZT - 1) / kZT));
        bp_global_kernel<TS, DIRECT><<<grid, kThreads, 0, st>>>(prm);
        return cudaGetLastError();
    }
    const size_t smem = sizeof(float) * (size_t)prm.J * prm.Rw * (prm.Wd + 1);
    cudaError_t e = ensure_smem<bp_generic_kernel<TS, DIRECT>>(smem);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)(nsq * prm.tps * prm.tps), (unsigned)((prm.nz + kZT - 1) / kZT));
    bp_generic_kernel<TS, DIRECT><<<grid, kThreads, smem, st>>>(prm);
    return cudaGetLastError();
}


// ---------------------------------------------------------------------------
// TMA path.  Same tiling and arithmetic as the generic kernel, but each
// view's window is one 3D bulk-tensor copy (zero fill outside the source),
// two stages of kViewsPerStage views are in flight (copy of stage c+1
// overlaps the gather of stage c), the per-view set-up is FP32 only, and the
// inner loop is
//   v = fma(1/U, i, v0);  fl = floor(v);  fv = v - fl;  one multiply-add for
//   the row address;  four shared loads at compile-time offsets;  two column
//   lerps pre-weighted by U^-2;  row lerp (about 18.7 instructions/update).
// Waits on the copies are bounded (FDKOD_ERR_TIMEOUT, then drain and exit).

struct BpTmaParams {
    float *vol;
    const GeomEntry *geo;
    const int32_t *crop;
    const int32_t *w0;
    int *status;
    int N, P, Nv, m, tps;
    int nviews, vstep, Pd;
    int RW, tile_stride;  // window rows; elements per staged window (128-byte multiple)
    int row0;             // detector row held in the source's row 0
    int zoff, nz;         // slices zoff .. zoff + nz - 1, written to vol[z - zoff]
    float scale;
    unsigned long long wait_ns;  // limit of every bounded wait (ns)
    int fault;                   // test hook (kTestFault*), 0 = none
};

// shared-memory load of one window element at a compile-time byte offset
// from a 32-bit address, widened to float32
template <typename TS, int OFF>
struct Lds;
template <int OFF>
struct Lds<float, OFF> {
    static __device__ __forceinline__ float f(uint32_t addr) {
        float v;
        asm volatile("ld.shared.f32 %0, [%1+%2];" : "=f"(v) : "r"(addr), "n"(OFF) : "memory");
        return v;
    }
};
template <int OFF>
struct Lds<__nv_bfloat16, OFF> {
    static __device__ __forceinline__ float f(uint32_t addr) {
        uint32_t u;
        asm volatile("ld.shared.u16 %0, [%1+%2];" : "=r"(u) : "r"(addr), "n"(OFF) : "memory");
        return __uint_as_float(u << 16);  // bfloat16 is the top half of a float32
    }
};
template <int OFF>
struct Lds<__half, OFF> {
    static __device__ __forceinline__ float f(uint32_t addr) {
        unsigned short h;
        asm volatile("ld.shared.u16 %0, [%1+%2];" : "=h"(h) : "r"(addr), "n"(OFF) : "memory");
        return __half2float(__ushort_as_half(h));
    }
};

// address bias: (row + kMagicBits) * 4 WD wraps to row * 4 WD in 32 bits once
// tbase absorbs -kMagicBits * 4 WD (keeps the unsigned arithmetic explicit)
constexpr int kMagicBits = 0x4B400000;
constexpr uint64_t kWaitLimitNs = 2000000000ull;
// test hooks of the failure paths (fdkod_set_test_fault)
constexpr int kTestFaultSkipCopy = 1;    // CTA 0 leaves out one copy of its chunk 1
constexpr int kTestFaultSmallWindow = 2; // every window counts as too small

// three CTAs per SM (the shared-memory limit): up to 80 registers per thread
template <typename TS, bool DIRECT, int WD>
__global__ void __launch_bounds__(kThreads, 3)
bp_tma_kernel(const __grid_constant__ CUtensorMap tmap, BpTmaParams a) {
    constexpr int ES = (int)sizeof(TS);      // window element size (bytes)
    constexpr int kAl = 16 / ES;             // copy start alignment (elements)
    extern __shared__ __align__(128) unsigned char smem_raw[];
    // 128-byte aligned staging area (offset from the shared array itself so
    // the compiler keeps shared-memory addressing)
    TS *sm = (TS *)(smem_raw + ((128u - (tma::smem_u32(smem_raw) & 127u)) & 127u));
    const uint32_t sbase = tma::smem_u32(sm);
    __shared__ __align__(8) uint64_t bars[2];
    __shared__ float4 s_pa[2][kViewsPerStage];  // cos, sin, 1/d_c, alpha
    __shared__ float4 s_pb[2][kViewsPerStage];  // gamma, g, column offset, row offset
    __shared__ float s_zcr[2][kViewsPerStage];  // z_c / d_c
    __shared__ int s_tx[2][kViewsPerStage], s_ty[2][kViewsPerStage], s_tz[2][kViewsPerStage];
    __shared__ int s_skip[2][kViewsPerStage];

    const int tiles = a.tps * a.tps;
    const int q = blockIdx.x / tiles;
    const int tt = blockIdx.x - q * tiles;
    const int qy = q / a.m, qx = q - qy * a.m;
    int ix0, ix1, iy0, iy1;
    square_range(qx, a.m, a.N, ix0, ix1);
    square_range(qy, a.m, a.N, iy0, iy1);
    const int x0 = ix0 + (tt % a.tps) * kTile;
    const int y0 = iy0 + (tt / a.tps) * kTile;
    if (x0 > ix1 || y0 > iy1) return;  // ragged square: empty tile (uniform per CTA)
    const int xe = min(x0 + kTile - 1, ix1), ye = min(y0 + kTile - 1, iy1);
    const int z0 = a.zoff + blockIdx.y * kZT;
    const int z1 = min(z0 + kZT - 1, a.zoff + a.nz - 1);

    const float half_n = 0.5f * (float)(a.N - 1);
    const float xc = 0.5f * ((float)ix0 + (float)ix1) - half_n;
    const float yc = 0.5f * ((float)iy0 + (float)iy1) - half_n;
    // centre of the full kZT-slice slab (also past the volume's end, so the
    // window always covers every slice the loop evaluates)
    const float zc = (float)z0 + 0.5f * (float)(kZT - 1) - half_n;
    const float vcd = 0.5f * (float)(a.Nv - 1);

    const int lx = threadIdx.x % kTile, ly = threadIdx.x / kTile;
    const int x = x0 + lx, y = y0 + ly;
    const bool active = x <= xe && y <= ye;
    const float dx = (float)x - half_n - xc, dy = (float)y - half_n - yc;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int32_t w0q = a.w0[q];
    const int nch = (a.nviews + kViewsPerStage - 1) / kViewsPerStage;

    // per-view window and coefficients of chunk c into stage st (warp w = view)
    auto setup = [&](int c, int st) {
        const int nj = min(kViewsPerStage, a.nviews - c * kViewsPerStage);
        if (warp < nj) {
            const int j = c * kViewsPerStage + warp;
            const int k = j * a.vstep;
            const size_t o = (size_t)q * a.P + k;
            const GeomEntry ge = a.geo[o];
            const int cbase = DIRECT ? a.crop[o] : 0;
            const float toff = DIRECT ? ge.frac - (float)w0q : -(float)w0q;
            const int cc = lane & 7;
            const float cx = (float)((cc & 1) ? xe : x0) - half_n - xc;
            const float cy = (float)((cc & 2) ? ye : y0) - half_n - yc;
            const float cz = (cc & 4) ? 0.5f * (float)(kZT - 1) : -0.5f * (float)(kZT - 1);
            const float dd = fmaf(ge.cb, cx, ge.sb * cy);
            const float invU = __fdividef(ge.g_hi, fmaf(ge.r, dd, 1.0f));
            const float t = fmaf(invU, fmaf(ge.alpha, cx, ge.gamma * cy), toff);
            const float zcr = zc * ge.r;
            // z_c g as hi + lo (exact product error by FMA)
            const float ph = zc * ge.g_hi;
            const float pl = fmaf(zc, ge.g_lo, fmaf(zc, ge.g_hi, -ph));
            const float v = (ph + vcd) + (pl + invU * (cz - zcr * dd));
            float tmin = t, tmax = t, vmin = v, vmax = v;
#pragma unroll
            for (int off = 4; off > 0; off >>= 1) {
                tmin = fminf(tmin, __shfl_xor_sync(0xffffffffu, tmin, off));
                tmax = fmaxf(tmax, __shfl_xor_sync(0xffffffffu, tmax, off));
                vmin = fminf(vmin, __shfl_xor_sync(0xffffffffu, vmin, off));
                vmax = fmaxf(vmax, __shfl_xor_sync(0xffffffffu, vmax, off));
            }
            if (lane == 0) {
                // columns read: floor(t) .. floor(t) + 1 over the tile, with one
                // sample of slack each side for FP32 rounding
                const int clo = cbase + (int)floorf(tmin) - 1;
                const int chi = cbase + (int)floorf(tmax) + 2;
                const int xs = clo & ~(kAl - 1);  // 16-byte aligned start of the copy
                const int vlo = (int)floorf(vmin) - 1;
                const int vhi = (int)floorf(vmax) + 2;
                const int skip =
                    (chi - xs > WD - 1) || (vhi - vlo > a.RW - 1) || a.fault == kTestFaultSmallWindow;
                if (skip) atomicOr(a.status, 1);
                s_pa[st][warp] = make_float4(ge.cb, ge.sb, ge.r, ge.alpha);
                s_pb[st][warp] = make_float4(ge.gamma, ge.g_hi, toff - (float)(xs - cbase),
                                             (ph - ((float)vlo - vcd)) + pl);
                s_zcr[st][warp] = zcr;
                s_tx[st][warp] = xs;
                s_ty[st][warp] = vlo - a.row0;  // row of the source (out of range: zero fill)
                s_tz[st][warp] = DIRECT ? k : q * a.Pd + j;
                s_skip[st][warp] = skip;
            }
        }
    };
    auto issue = [&](int c, int st) {
        const int nj = min(kViewsPerStage, a.nviews - c * kViewsPerStage);
        tma::fence_proxy_async();
        tma::mbar_arrive_expect_tx(&bars[st], (uint32_t)(nj * a.RW * WD * ES));
        for (int w = 0; w < nj; ++w) {
            // test hook: the stage's bytes never all arrive, its wait runs out
            if (a.fault == kTestFaultSkipCopy && c == 1 && w == 0 && blockIdx.x == 0 && blockIdx.y == 0) continue;
            tma::load_3d(sm + (size_t)(st * kViewsPerStage + w) * a.tile_stride, &tmap, &bars[st], s_tx[st][w],
                         s_ty[st][w], s_tz[st][w]);
        }
    };

    if (threadIdx.x == 0) {
        tma::mbar_init(&bars[0], 1);
        tma::mbar_init(&bars[1], 1);
        tma::fence_mbar_init();
    }
    __syncthreads();
    setup(0, 0);
    __syncthreads();
    if (threadIdx.x == 0) issue(0, 0);

    float acc[kZT];
#pragma unroll
    for (int i = 0; i < kZT; ++i) acc[i] = 0.f;

    for (int c = 0; c < nch; ++c) {
        const int st = c & 1;
        if (c + 1 < nch) setup(c + 1, st ^ 1);
        __syncthreads();
        if (c + 1 < nch && threadIdx.x == 0) issue(c + 1, st ^ 1);
        const bool ok = tma::mbar_wait_bounded(&bars[st], (uint32_t)((c >> 1) & 1), a.wait_ns);
        if (!__syncthreads_and(ok)) {
            // a copy never completed: report, let copies in flight land, leave
            if (threadIdx.x == 0) atomicOr(a.status, 2);
            tma::mbar_wait_bounded(&bars[st], (uint32_t)((c >> 1) & 1), a.wait_ns);
            if (c + 1 < nch) tma::mbar_wait_bounded(&bars[st ^ 1], (uint32_t)(((c + 1) >> 1) & 1), a.wait_ns);
            return;
        }
        if (active) {
            const int nj = min(kViewsPerStage, a.nviews - c * kViewsPerStage);
            for (int w = 0; w < nj; ++w) {
                if (s_skip[st][w]) continue;
                const float4 pa = s_pa[st][w];
                const float4 pb = s_pb[st][w];
                const float dd = fmaf(pa.x, dx, pa.y * dy);
                const float invU = __fdividef(pb.y, fmaf(pa.z, dd, 1.0f));
                const float t = fmaf(invU, fmaf(pa.w, dx, pb.x * dy), pb.z);
                const float tf = floorf(t);
                const float wgt = invU * invU;
                const float a1 = wgt * (t - tf);
                const float a0 = wgt - a1;
                const float vb0 = fmaf(invU, -0.5f * (float)(kZT - 1) - s_zcr[st][w] * dd, pb.w);
                // 32-bit shared address of sample (row 0, column floor(t));
                // the row offset folds into one multiply-add per slice
                const uint32_t tbase = sbase + (uint32_t)ES * ((uint32_t)(st * kViewsPerStage + w) *
                                                                    (uint32_t)a.tile_stride + (uint32_t)(int)tf) -
                                       (uint32_t)kMagicBits * (uint32_t)(ES * WD);
#pragma unroll
                for (int i = 0; i < kZT; ++i) {
                    const float v = fmaf(invU, (float)i, vb0);
                    const float fl = floorf(v);
                    const float fv = v - fl;
                    const uint32_t ad = (uint32_t)((int)fl + kMagicBits) * (uint32_t)(ES * WD) + tbase;
                    const float c0 = fmaf(a1, Lds<TS, ES>::f(ad), a0 * Lds<TS, 0>::f(ad));
                    const float c1 = fmaf(a1, Lds<TS, ES * WD + ES>::f(ad), a0 * Lds<TS, ES * WD>::f(ad));
                    acc[i] = fmaf(fv, c1 - c0, acc[i] + c0);
                }
            }
        }
        __syncthreads();
    }
    if (active) {
#pragma unroll
        for (int i = 0; i < kZT; ++i)
            if (z0 + i <= z1) a.vol[((size_t)(z0 + i - a.zoff) * a.N + y) * a.N + x] = acc[i] * a.scale;
    }
}

// ---------------------------------------------------------------------------
// Mirrored-pair form of the staged backprojection (whole volumes).  Each
// thread owns kZP slices p0 .. p0 + kZP - 1 of the lower half of its (x, y)
// column and their mirror images N - 1 - p about the mid-plane z = 0.  A
// voxel and its mirror read the same column (Eq. 1 does not involve z) and
// mirrored rows: z/U + (Nv-1)/2 and -z/U + (Nv-1)/2 add up to Nv - 1.  So
// the column weights, the row fraction and the per-view set-up are shared
// by the pair, and with the two windows of a view staged at row origins vlo
// and vlo', the mirror's window row is C - v for C = Nv - 1 - vlo - vlo'.
// Row coordinates are 9.23 fixed point: v = V 2^-23 advances by an integer
// step per slice, the row is V >> 23 and the fraction's float is the
// mantissa bits of V under the exponent of 1.0.  Where every thread of a
// warp has 1/U <= 1 for the view, consecutive slices move by 0 or 1 row,
// so each slice loads only its new row of the pair (two samples per voxel
// instead of four) and keeps the other from the previous slice.
struct BpPairParams {
    float *vol;
    const GeomEntry *geo;
    const int32_t *crop;
    const int32_t *w0;
    int *status;
    int N, P, Nv, m, tps;
    int nviews, vstep, Pd;
    int RW, tile_stride;  // rows of a kZP-slice window; elements per staged window
    int pbase, pend;      // slice pairs pbase .. pend - 1 (pair p: slices p and N - 1 - p)
    float scale;
    unsigned long long wait_ns;
    int fault;
};

// Warp-specialised: warp 8 is the producer (per chunk of VPS views it finds
// the windows, writes the view parameters and issues the copies into a ring
// of kPairSlots slots); warps 0-7 consume.  A slot is full when its copies
// have landed (full[slot], which also publishes the producer's parameters)
// and free again when all eight consumer warps have arrived on empty[slot]:
// no block-wide barrier inside the view loop, so consumer warps drift within
// the ring instead of waiting for the slowest.  Every wait is bounded
// (FDKOD_ERR_TIMEOUT); a producer that gives up waits for its copies in
// flight before it leaves.  The producer polls `empty` (mbarrier.test_wait):
// suspended in mbarrier.try_wait it was measured to resume late (the whole
// kernel 1.4x slower); the consumers' waits on `full` are mostly satisfied
// at once and suspend (polling them measured no faster).
constexpr int kPairSlots = 3;
constexpr int kPairConsumers = kThreads / 32;      // 8
constexpr int kPairThreads = kThreads + 32;        // plus the producer warp

template <typename TS, bool DIRECT, int WD, int VPS>
__global__ void __launch_bounds__(kPairThreads, 3)
bp_pair_kernel(const __grid_constant__ CUtensorMap tmap, BpPairParams a) {
    constexpr int ES = (int)sizeof(TS);
    constexpr int kAl = 16 / ES;
    constexpr uint32_t ROWB = (uint32_t)(ES * WD);  // bytes per window row
    constexpr float kFix = 8388608.0f;              // 2^23
    static_assert(VPS * 16 <= 32, "the producer warp sets up VPS views at 16 lanes each");
    extern __shared__ __align__(128) unsigned char smem_raw[];
    TS *sm = (TS *)(smem_raw + ((128u - (tma::smem_u32(smem_raw) & 127u)) & 127u));
    const uint32_t sbase = tma::smem_u32(sm);
    __shared__ __align__(8) uint64_t full[kPairSlots], empty[kPairSlots];
    __shared__ float4 s_pa[kPairSlots][VPS];  // cos, sin, 1/d_c, alpha
    __shared__ float4 s_pb[kPairSlots][VPS];  // gamma, g, column offset, window row of the lower slab's centre
    __shared__ float s_zcr[kPairSlots][VPS];  // z_c / d_c (lower slab)
    __shared__ int s_C[kPairSlots][VPS], s_skip[kPairSlots][VPS];

    const int tiles = a.tps * a.tps;
    const int q = blockIdx.x / tiles;
    const int tt = blockIdx.x - q * tiles;
    const int qy = q / a.m, qx = q - qy * a.m;
    int ix0, ix1, iy0, iy1;
    square_range(qx, a.m, a.N, ix0, ix1);
    square_range(qy, a.m, a.N, iy0, iy1);
    const int x0 = ix0 + (tt % a.tps) * kTile;
    const int y0 = iy0 + (tt / a.tps) * kTile;
    if (x0 > ix1 || y0 > iy1) return;  // ragged square: empty tile (uniform per CTA)
    const int xe = min(x0 + kTile - 1, ix1), ye = min(y0 + kTile - 1, iy1);
    const int p0 = a.pbase + blockIdx.y * kZP;  // first slice pair

    const float half_n = 0.5f * (float)(a.N - 1);
    const float xc = 0.5f * ((float)ix0 + (float)ix1) - half_n;
    const float yc = 0.5f * ((float)iy0 + (float)iy1) - half_n;
    // centre of the lower slab (the upper one is centred at -zc)
    const float zc = (float)p0 + 0.5f * (float)(kZP - 1) - half_n;
    const float vcd = 0.5f * (float)(a.Nv - 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nch = (a.nviews + VPS - 1) / VPS;
    // window of view w of slot sl, lower (h = 0) or upper (h = 1) slab
    auto win = [&](int sl, int w, int h) { return (uint32_t)((sl * VPS + w) * 2 + h) * (uint32_t)a.tile_stride; };

    if (threadIdx.x == 0) {
        for (int i = 0; i < kPairSlots; ++i) {
            tma::mbar_init(&full[i], 1);
            tma::mbar_init(&empty[i], kPairConsumers);
        }
        tma::fence_mbar_init();
    }
    __syncthreads();

    if (warp == kPairConsumers) {
        // ---- producer: lanes 16 w .. 16 w + 15 set up view w of the chunk,
        // 0-7 of them at the corners of the lower slab, 8-15 of the upper
        const int32_t w0q = a.w0[q];
        const int w = lane >> 4, cc = lane & 7;
        const float zcl = (lane & 8) ? -zc : zc;
        const float cx = (float)((cc & 1) ? xe : x0) - half_n - xc;
        const float cy = (float)((cc & 2) ? ye : y0) - half_n - yc;
        const float cz = (cc & 4) ? 0.5f * (float)(kZP - 1) : -0.5f * (float)(kZP - 1);
        int c = 0;
        for (; c < nch; ++c) {
            const int sl = c % kPairSlots;
            // round r of a slot may start once its round r - 1 was consumed
            // (lane 0 waits; the warp follows its answer)
            bool ok = true;
            if (c >= kPairSlots && lane == 0)
                ok = tma::mbar_wait_spin(&empty[sl], (uint32_t)(((c / kPairSlots) & 1) ^ 1), a.wait_ns);
            if (!__shfl_sync(0xffffffffu, ok, 0)) {
                if (lane == 0) atomicOr(a.status, 2);
                break;
            }
            const int nj = min(VPS, a.nviews - c * VPS);
            const int j = c * VPS + min(w, nj - 1);  // lanes past the chunk repeat its last view
            const int k = j * a.vstep;
            const size_t o = (size_t)q * a.P + k;
            const GeomEntry ge = a.geo[o];
            const int cbase = DIRECT ? a.crop[o] : 0;
            const float toff = DIRECT ? ge.frac - (float)w0q : -(float)w0q;
            const float dd = fmaf(ge.cb, cx, ge.sb * cy);
            const float invU = __fdividef(ge.g_hi, fmaf(ge.r, dd, 1.0f));
            const float t = fmaf(invU, fmaf(ge.alpha, cx, ge.gamma * cy), toff);
            const float zcr = zcl * ge.r;
            // z_c g as hi + lo (exact product error by FMA)
            const float ph = zcl * ge.g_hi;
            const float pl = fmaf(zcl, ge.g_lo, fmaf(zcl, ge.g_hi, -ph));
            const float v = (ph + vcd) + (pl + invU * (cz - zcr * dd));
            float tmin = t, tmax = t, vmin = v, vmax = v;
#pragma unroll
            for (int off = 4; off > 0; off >>= 1) {  // within each half's 8 corners
                vmin = fminf(vmin, __shfl_xor_sync(0xffffffffu, vmin, off));
                vmax = fmaxf(vmax, __shfl_xor_sync(0xffffffffu, vmax, off));
            }
#pragma unroll
            for (int off = 8; off > 0; off >>= 1) {  // columns: both halves
                tmin = fminf(tmin, __shfl_xor_sync(0xffffffffu, tmin, off));
                tmax = fmaxf(tmax, __shfl_xor_sync(0xffffffffu, tmax, off));
            }
            const float vmin2 = __shfl_down_sync(0xffffffffu, vmin, 8);
            const float vmax2 = __shfl_down_sync(0xffffffffu, vmax, 8);
            // lane 16 w: columns read floor(t) .. floor(t) + 1 over the tile,
            // one sample of slack each side for FP32 rounding
            const int clo = cbase + (int)floorf(tmin) - 1;
            const int chi = cbase + (int)floorf(tmax) + 2;
            const int xs = clo & ~(kAl - 1);  // 16-byte aligned start of the copy
            const int vlo = (int)floorf(vmin) - 1, vhi = (int)floorf(vmax) + 2;
            const int vlo2 = (int)floorf(vmin2) - 1, vhi2 = (int)floorf(vmax2) + 2;
            const bool lead = (lane & 15) == 0 && w < nj;
            if (lead) {
                const int skip = (chi - xs > WD - 1) || (vhi - vlo > a.RW - 1) || (vhi2 - vlo2 > a.RW - 1) ||
                                 a.fault == kTestFaultSmallWindow;
                if (skip) atomicOr(a.status, 1);
                s_pa[sl][w] = make_float4(ge.cb, ge.sb, ge.r, ge.alpha);
                s_pb[sl][w] = make_float4(ge.gamma, ge.g_hi, toff - (float)(xs - cbase), (ph - ((float)vlo - vcd)) + pl);
                s_zcr[sl][w] = zcr;
                s_C[sl][w] = (a.Nv - 1) - vlo - vlo2;
                s_skip[sl][w] = skip;
            }
            // the copies: lane 0 for every view of the chunk
            const int xs0 = __shfl_sync(0xffffffffu, xs, 0), xs1 = __shfl_sync(0xffffffffu, xs, 16);
            const int vl0 = __shfl_sync(0xffffffffu, vlo, 0), vl1 = __shfl_sync(0xffffffffu, vlo, 16);
            const int vu0 = __shfl_sync(0xffffffffu, vlo2, 0), vu1 = __shfl_sync(0xffffffffu, vlo2, 16);
            const int tz = DIRECT ? k : q * a.Pd + j;
            const int tz0 = __shfl_sync(0xffffffffu, tz, 0), tz1 = __shfl_sync(0xffffffffu, tz, 16);
            __syncwarp();  // the parameters are written before lane 0 publishes them
            if (lane == 0) {
                tma::fence_proxy_async();
                tma::mbar_arrive_expect_tx(&full[sl], (uint32_t)(nj * 2 * a.RW * WD * ES));
                for (int v2 = 0; v2 < nj; ++v2) {
                    // test hook: the slot's bytes never all arrive, its wait runs out
                    if (a.fault == kTestFaultSkipCopy && c == 1 && v2 == 0 && blockIdx.x == 0 && blockIdx.y == 0)
                        continue;
                    const int x = v2 == 0 ? xs0 : xs1, z = v2 == 0 ? tz0 : tz1;
                    tma::load_3d(sm + win(sl, v2, 0), &tmap, &full[sl], x, v2 == 0 ? vl0 : vl1, z);
                    tma::load_3d(sm + win(sl, v2, 1), &tmap, &full[sl], x, v2 == 0 ? vu0 : vu1, z);
                }
            }
            __syncwarp();
        }
        // copies still in flight must land before the CTA may exit
        if (lane == 0)
            for (int m = max(0, c - kPairSlots); m < c; ++m)
                tma::mbar_wait_bounded(&full[m % kPairSlots], (uint32_t)((m / kPairSlots) & 1), a.wait_ns);
        return;
    }

    // ---- consumers.  A voxel and its mirror go through the same operations
    // on different samples, so they share packed two-lane FP32 instructions
    // (x: lower slab, y: upper slab; each lane rounds as the scalar
    // operation would): half the arithmetic instructions of two scalar
    // updates.
    const int lx = threadIdx.x % kTile, ly = threadIdx.x / kTile;
    const int x = x0 + lx, y = y0 + ly;
    const bool active = x <= xe && y <= ye;
    const float dx = (float)x - half_n - xc, dy = (float)y - half_n - yc;
    float2 acc[kZP];  // (lower slab, upper mirrored slab)
#pragma unroll
    for (int i = 0; i < kZP; ++i) acc[i] = make_float2(0.f, 0.f);

    for (int c = 0; c < nch; ++c) {
        const int sl = c % kPairSlots;
        const bool ok = tma::mbar_wait_bounded(&full[sl], (uint32_t)((c / kPairSlots) & 1), a.wait_ns);
        if (!__all_sync(0xffffffffu, ok)) {
            if (lane == 0) atomicOr(a.status, 2);
            return;  // the producer waits for the copies in flight
        }
        const int nj = min(VPS, a.nviews - c * VPS);
        for (int w = 0; w < nj; ++w) {
            if (s_skip[sl][w]) continue;  // uniform per CTA
            const float4 pa = s_pa[sl][w];
            const float4 pb = s_pb[sl][w];
            const float dd = fmaf(pa.x, dx, pa.y * dy);
            const float invU = __fdividef(pb.y, fmaf(pa.z, dd, 1.0f));
            const uint32_t dV = __float2uint_rn(invU * kFix);
            // warp-uniform choice (threads outside a ragged tile do not constrain it)
            const bool stepA = __all_sync(0xffffffffu, !active || dV <= (1u << 23));
            if (!active) continue;
            const float t = fmaf(invU, fmaf(pa.w, dx, pb.x * dy), pb.z);
            const float tf = floorf(t);
            const float wgt = invU * invU;
            const float a1 = wgt * (t - tf);
            const float a0 = wgt - a1;
            const float2 A1 = make_float2(a1, a1), A0 = make_float2(a0, a0);
            // window row of slice p0 (lower slab), in 9.23 fixed point
            const float vb0 = fmaf(invU, -0.5f * (float)(kZP - 1) - s_zcr[sl][w] * dd, pb.w);
            uint32_t V = __float2uint_rn(vb0 * kFix);
            // byte addresses: row r of the lower window at r ROWB + bL; the
            // upper window's row C - 1 - r at KLU - (r ROWB + bL)
            const uint32_t bL = sbase + (uint32_t)ES * (win(sl, w, 0) + (uint32_t)(int)tf);
            const uint32_t bU = sbase + (uint32_t)ES * (win(sl, w, 1) + (uint32_t)(int)tf);
            const uint32_t KLU = (uint32_t)(s_C[sl][w] - 1) * ROWB + bU + bL;
            // column-interpolated samples (U^-2 weighted) of the pair's first
            // row (lower row r, upper row C - r) and of its second row
            auto first = [&](uint32_t aL, uint32_t aU) {
                return __ffma2_rn(A1, make_float2(Lds<TS, ES>::f(aL), Lds<TS, ROWB + ES>::f(aU)),
                                  __fmul2_rn(A0, make_float2(Lds<TS, 0>::f(aL), Lds<TS, ROWB>::f(aU))));
            };
            auto second = [&](uint32_t aL, uint32_t aU) {
                return __ffma2_rn(A1, make_float2(Lds<TS, ROWB + ES>::f(aL), Lds<TS, ES>::f(aU)),
                                  __fmul2_rn(A0, make_float2(Lds<TS, ROWB>::f(aL), Lds<TS, 0>::f(aU))));
            };
            // row weights 1 - f and f (both lanes) from the fixed-point row
            // coordinate: fb = 1 + f exactly, so 2 - fb and fb - 1 are exact
            auto rowlerp = [&](uint32_t Vc, float2 A, float2 B, float2 acc_i) {
                const float fb = __uint_as_float((Vc & 0x7fffffu) | 0x3f800000u);
                const float f = fb - 1.0f, g = 2.0f - fb;
                return __ffma2_rn(make_float2(f, f), B, __ffma2_rn(make_float2(g, g), A, acc_i));
            };
            if (stepA) {
                // 1/U <= 1: the row advances by 0 or 1 per slice
                uint32_t r = V >> 23;
                uint32_t aL = r * ROWB + bL, aU = KLU - aL;
                float2 A = first(aL, aU);
                float2 B = second(aL, aU);
                acc[0] = rowlerp(V, A, B, acc[0]);
#pragma unroll
                for (int i = 1; i < kZP; ++i) {
                    V += dV;
                    const uint32_t rn = V >> 23;
                    const bool adv = rn != r;
                    r = rn;
                    aL = r * ROWB + bL;
                    aU = KLU - aL;
                    A = adv ? B : A;
                    B = second(aL, aU);
                    acc[i] = rowlerp(V, A, B, acc[i]);
                }
            } else {
#pragma unroll
                for (int i = 0; i < kZP; ++i) {
                    const uint32_t r = V >> 23;
                    const uint32_t aL = r * ROWB + bL, aU = KLU - aL;
                    const float2 A = first(aL, aU);
                    const float2 B = second(aL, aU);
                    acc[i] = rowlerp(V, A, B, acc[i]);
                    V += dV;
                }
            }
        }
        __syncwarp();
        if (lane == 0) tma::mbar_arrive(&empty[sl]);  // this warp is done with the slot
    }
    if (active) {
#pragma unroll
        for (int i = 0; i < kZP; ++i) {
            const int pz = p0 + i;
            if (pz < a.pend) {
                const int zu = a.N - 1 - pz;
                a.vol[((size_t)pz * a.N + y) * a.N + x] = acc[i].x * a.scale;
                if (zu != pz) a.vol[((size_t)zu * a.N + y) * a.N + x] = acc[i].y * a.scale;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Persistent form for a batch of plans (float32 windows): one launch, as
// many CTAs as fit the GPU, each taking work items (plan, tile, z-slab) from
// an atomic counter until the list is exhausted; per item the arithmetic of
// bp_tma_kernel, with the plan's tensor map and parameters read from global
// memory and the window width a run-time value (the second window row is one
// add away).  The mbarrier stages continue from item to item.
struct BatchInst {
    BpTmaParams a;
    int direct, WD;
};

__global__ void __launch_bounds__(kThreads, 3)
bp_persistent_kernel(const CUtensorMap *__restrict__ maps, const BatchInst *__restrict__ insts,
                     const int4 *__restrict__ items, int nitems, int *counter) {
    constexpr int kAl = 4;  // float windows: 16-byte copy alignment in elements
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float *sm = (float *)(smem_raw + ((128u - (tma::smem_u32(smem_raw) & 127u)) & 127u));
    const uint32_t sbase = tma::smem_u32(sm);
    __shared__ __align__(8) uint64_t bars[2];
    __shared__ float4 s_pa[2][kViewsPerStage];
    __shared__ float4 s_pb[2][kViewsPerStage];
    __shared__ float s_zcr[2][kViewsPerStage];
    __shared__ int s_tx[2][kViewsPerStage], s_ty[2][kViewsPerStage], s_tz[2][kViewsPerStage];
    __shared__ int s_skip[2][kViewsPerStage];
    __shared__ int s_item;
    if (threadIdx.x == 0) {
        tma::mbar_init(&bars[0], 1);
        tma::mbar_init(&bars[1], 1);
        tma::fence_mbar_init();
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint32_t gc = 0;  // chunks this CTA has run: stage gc % 2, parity (gc / 2) % 2

    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
        __syncthreads();
        const int item = s_item;
        __syncthreads();
        if (item >= nitems) break;
        const int4 it = items[item];  // plan, tile, z-slab
        const BpTmaParams a = insts[it.x].a;
        const bool direct = insts[it.x].direct != 0;
        const int WD = insts[it.x].WD;
        const CUtensorMap *map = maps + it.x;

        const int tiles = a.tps * a.tps;
        const int q = it.y / tiles;
        const int tt = it.y - q * tiles;
        const int qy = q / a.m, qx = q - qy * a.m;
        int ix0, ix1, iy0, iy1;
        square_range(qx, a.m, a.N, ix0, ix1);
        square_range(qy, a.m, a.N, iy0, iy1);
        const int x0 = ix0 + (tt % a.tps) * kTile;
        const int y0 = iy0 + (tt / a.tps) * kTile;
        if (x0 > ix1 || y0 > iy1) continue;  // ragged square: empty tile (uniform)
        const int xe = min(x0 + kTile - 1, ix1), ye = min(y0 + kTile - 1, iy1);
        const int z0 = a.zoff + it.z * kZT;
        const int z1 = min(z0 + kZT - 1, a.zoff + a.nz - 1);
        const float half_n = 0.5f * (float)(a.N - 1);
        const float xc = 0.5f * ((float)ix0 + (float)ix1) - half_n;
        const float yc = 0.5f * ((float)iy0 + (float)iy1) - half_n;
        const float zc = (float)z0 + 0.5f * (float)(kZT - 1) - half_n;
        const float vcd = 0.5f * (float)(a.Nv - 1);
        const int lx = threadIdx.x % kTile, ly = threadIdx.x / kTile;
        const int x = x0 + lx, y = y0 + ly;
        const bool active = x <= xe && y <= ye;
        const float dx = (float)x - half_n - xc, dy = (float)y - half_n - yc;
        const int32_t w0q = a.w0[q];
        const int nch = (a.nviews + kViewsPerStage - 1) / kViewsPerStage;

        auto setup = [&](int c, int st) {
            const int nj = min(kViewsPerStage, a.nviews - c * kViewsPerStage);
            if (warp < nj) {
                const int j = c * kViewsPerStage + warp;
                const int k = j * a.vstep;
                const size_t o = (size_t)q * a.P + k;
                const GeomEntry ge = a.geo[o];
                const int cbase = direct ? a.crop[o] : 0;
                const float toff = direct ? ge.frac - (float)w0q : -(float)w0q;
                const int cc = lane & 7;
                const float cx = (float)((cc & 1) ? xe : x0) - half_n - xc;
                const float cy = (float)((cc & 2) ? ye : y0) - half_n - yc;
                const float cz = (cc & 4) ? 0.5f * (float)(kZT - 1) : -0.5f * (float)(kZT - 1);
                const float dd = fmaf(ge.cb, cx, ge.sb * cy);
                const float invU = __fdividef(ge.g_hi, fmaf(ge.r, dd, 1.0f));
                const float t = fmaf(invU, fmaf(ge.alpha, cx, ge.gamma * cy), toff);
                const float zcr = zc * ge.r;
                const float ph = zc * ge.g_hi;
                const float pl = fmaf(zc, ge.g_lo, fmaf(zc, ge.g_hi, -ph));
                const float v = (ph + vcd) + (pl + invU * (cz - zcr * dd));
                float tmin = t, tmax = t, vmin = v, vmax = v;
#pragma unroll
                for (int off = 4; off > 0; off >>= 1) {
                    tmin = fminf(tmin, __shfl_xor_sync(0xffffffffu, tmin, off));
                    tmax = fmaxf(tmax, __shfl_xor_sync(0xffffffffu, tmax, off));
                    vmin = fminf(vmin, __shfl_xor_sync(0xffffffffu, vmin, off));
                    vmax = fmaxf(vmax, __shfl_xor_sync(0xffffffffu, vmax, off));
                }
                if (lane == 0) {
                    const int clo = cbase + (int)floorf(tmin) - 1;
                    const int chi = cbase + (int)floorf(tmax) + 2;
                    const int xs = clo & ~(kAl - 1);
                    const int vlo = (int)floorf(vmin) - 1;
                    const int vhi = (int)floorf(vmax) + 2;
                    const int skip = (chi - xs > WD - 1) || (vhi - vlo > a.RW - 1);
                    if (skip) atomicOr(a.status, 1);
                    s_pa[st][warp] = make_float4(ge.cb, ge.sb, ge.r, ge.alpha);
                    s_pb[st][warp] = make_float4(ge.gamma, ge.g_hi, toff - (float)(xs - cbase),
                                                 (ph - ((float)vlo - vcd)) + pl);
                    s_zcr[st][warp] = zcr;
                    s_tx[st][warp] = xs;
                    s_ty[st][warp] = vlo - a.row0;
                    s_tz[st][warp] = direct ? k : q * a.Pd + j;
                    s_skip[st][warp] = skip;
                }
            }
        };
        auto issue = [&](int c, int st) {
            const int nj = min(kViewsPerStage, a.nviews - c * kViewsPerStage);
            tma::fence_proxy_async();
            tma::mbar_arrive_expect_tx(&bars[st], (uint32_t)(nj * a.RW * WD * 4));
            for (int w = 0; w < nj; ++w)
                tma::load_3d(sm + (size_t)(st * kViewsPerStage + w) * a.tile_stride, map, &bars[st], s_tx[st][w],
                             s_ty[st][w], s_tz[st][w]);
        };

        setup(0, (int)(gc & 1u));
        __syncthreads();
        if (threadIdx.x == 0) issue(0, (int)(gc & 1u));
        float acc[kZT];
#pragma unroll
        for (int i = 0; i < kZT; ++i) acc[i] = 0.f;
        const uint32_t rowb = 4u * (uint32_t)WD;
        for (int c = 0; c < nch; ++c) {
            const uint32_t g = gc + (uint32_t)c;
            const int st = (int)(g & 1u);
            if (c + 1 < nch) setup(c + 1, st ^ 1);
            __syncthreads();
            if (c + 1 < nch && threadIdx.x == 0) issue(c + 1, st ^ 1);
            const bool ok = tma::mbar_wait_bounded(&bars[st], (g >> 1) & 1u, kWaitLimitNs);
            if (!__syncthreads_and(ok)) {
                if (threadIdx.x == 0) atomicOr(a.status, 2);
                tma::mbar_wait_bounded(&bars[st], (g >> 1) & 1u, kWaitLimitNs);
                if (c + 1 < nch) tma::mbar_wait_bounded(&bars[st ^ 1], ((g + 1) >> 1) & 1u, kWaitLimitNs);
                return;
            }
            if (active) {
                const int nj = min(kViewsPerStage, a.nviews - c * kViewsPerStage);
                for (int w = 0; w < nj; ++w) {
                    if (s_skip[st][w]) continue;
                    const float4 pa = s_pa[st][w];
                    const float4 pb = s_pb[st][w];
                    const float dd = fmaf(pa.x, dx, pa.y * dy);
                    const float invU = __fdividef(pb.y, fmaf(pa.z, dd, 1.0f));
                    const float t = fmaf(invU, fmaf(pa.w, dx, pb.x * dy), pb.z);
                    const float tf = floorf(t);
                    const float wgt = invU * invU;
                    const float a1 = wgt * (t - tf);
                    const float a0 = wgt - a1;
                    const float vb0 = fmaf(invU, -0.5f * (float)(kZT - 1) - s_zcr[st][w] * dd, pb.w);
                    const uint32_t tbase = sbase + 4u * ((uint32_t)(st * kViewsPerStage + w) *
                                                             (uint32_t)a.tile_stride + (uint32_t)(int)tf) -
                                           (uint32_t)kMagicBits * rowb;
#pragma unroll
                    for (int i = 0; i < kZT; ++i) {
                        const float v = fmaf(invU, (float)i, vb0);
                        const float fl = floorf(v);
                        const float fv = v - fl;
                        const uint32_t ad = (uint32_t)((int)fl + kMagicBits) * rowb + tbase;
                        const uint32_t ad2 = ad + rowb;
                        const float c0 = fmaf(a1, Lds<float, 4>::f(ad), a0 * Lds<float, 0>::f(ad));
                        const float c1 = fmaf(a1, Lds<float, 4>::f(ad2), a0 * Lds<float, 0>::f(ad2));
                        acc[i] = fmaf(fv, c1 - c0, acc[i] + c0);
                    }
                }
            }
            __syncthreads();
        }
        gc += (uint32_t)nch;
        if (active) {
#pragma unroll
            for (int i = 0; i < kZT; ++i)
                if (z0 + i <= z1) a.vol[((size_t)(z0 + i - a.zoff) * a.N + y) * a.N + x] = acc[i] * a.scale;
        }
    }
}

template <typename TS, bool DIRECT, int WD>
cudaError_t launch_tma_t(const CUtensorMap &map, const BpTmaParams &prm, int nsq, cudaStream_t st) {
    const size_t smem = sizeof(TS) * (size_t)2 * kViewsPerStage * prm.tile_stride + 128;
    cudaError_t e = ensure_smem<bp_tma_kernel<TS, DIRECT, WD>>(smem);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)(nsq * prm.tps * prm.tps), (unsigned)((prm.nz + kZT - 1) / kZT));
    bp_tma_kernel<TS, DIRECT, WD><<<grid, kThreads, smem, st>>>(map, prm);
    return cudaGetLastError();
}

template <typename TS, bool DIRECT>
cudaError_t launch_tma_w(int WD, const CUtensorMap &map, const BpTmaParams &prm, int nsq, cudaStream_t st) {
    switch (WD) {
        case 32: return launch_tma_t<TS, DIRECT, 32>(map, prm, nsq, st);
        case 48: return launch_tma_t<TS, DIRECT, 48>(map, prm, nsq, st);
        case 64: return launch_tma_t<TS, DIRECT, 64>(map, prm, nsq, st);
        case 96: return launch_tma_t<TS, DIRECT, 96>(map, prm, nsq, st);
        case 128: return launch_tma_t<TS, DIRECT, 128>(map, prm, nsq, st);
    }
    return cudaErrorInvalidValue;
}

// The TMA path applies when the source is 16-byte aligned, its rows are whole
// 16-byte units, and the window fits a box (<= 256 rows, width an
// instantiated WD).  The decomposed data is float32; Q may be 16-bit.
// Fills the tensor map, the parameters and the window width; false when the
// TMA path does not apply.
bool make_tma_launch(const PlanImpl &p, const SquareSet &ss, bool direct, const void *src, float *vol,
                     const Band &b, CUtensorMap &map, BpTmaParams &a, int &WD) {
    const int es = (direct && p.qtype != FDKOD_F32) ? 2 : 4;
    WD = es == 4 ? ss.WdT : ss.WdT16;
    if (WD == 0 || ss.Rw > 256 || ((uintptr_t)src & 15) != 0) return false;
    if (direct && ((size_t)p.g.Nu * es) % 16 != 0) return false;
    uint64_t dims[3], strides[2];
    if (direct) {
        dims[0] = (uint64_t)p.g.Nu;
        dims[1] = (uint64_t)b.nrows;
        dims[2] = (uint64_t)p.g.P;
        strides[0] = (uint64_t)p.g.Nu * es;
    } else {
        dims[0] = (uint64_t)p.Tstride;
        dims[1] = (uint64_t)b.nrows;
        dims[2] = (uint64_t)ss.nsq * p.Pd;
        strides[0] = (uint64_t)p.Tstride * sizeof(float);
    }
    strides[1] = strides[0] * dims[1];
    const uint32_t box[3] = {(uint32_t)WD, (uint32_t)ss.Rw, 1u};
    const CUtensorMapDataType dt = es == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                   : (p.qtype == FDKOD_F16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                                           : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16);
    if (encode_map_3d(&map, dt, src, dims, strides, box) != cudaSuccess) return false;  // generic path
    a = BpTmaParams{};
    a.vol = vol;
    a.geo = ss.geo;
    a.crop = ss.crop;
    a.w0 = ss.w0;
    a.status = p.status;
    a.N = p.g.N;
    a.P = p.g.P;
    a.Nv = p.g.Nv;
    a.m = ss.m;
    a.tps = ss.tiles_per_side;
    a.Pd = p.Pd;
    a.RW = ss.Rw;
    a.row0 = b.row0;
    a.zoff = b.zoff;
    a.nz = b.nz;
    a.wait_ns = p.wait_ns > 0 ? (unsigned long long)p.wait_ns : kWaitLimitNs;
    a.fault = p.test_fault;
    // elements per staged window, a 128-byte multiple
    a.tile_stride = (ss.Rw * WD + (128 / es - 1)) & ~(128 / es - 1);
    if (direct) {
        a.nviews = p.g.P;
        a.vstep = 1;
        a.scale = (float)(M_PI / (double)p.g.P);
    } else {
        a.nviews = p.Pd;
        a.vstep = p.D;
        a.scale = (float)(M_PI / (double)p.Pd);
    }
    return true;
}

cudaError_t try_launch_tma(const PlanImpl &p, const SquareSet &ss, bool direct, const void *src, float *vol,
                           cudaStream_t st, const Band &b, bool &launched) {
    launched = false;
    CUtensorMap map;
    BpTmaParams a;
    int WD = 0;
    if (!make_tma_launch(p, ss, direct, src, vol, b, map, a, WD)) return cudaSuccess;
    launched = true;
    if (!direct) return launch_tma_w<float, false>(WD, map, a, ss.nsq, st);
    switch (p.qtype) {
        case FDKOD_F32: return launch_tma_w<float, true>(WD, map, a, ss.nsq, st);
        case FDKOD_BF16: return launch_tma_w<__nv_bfloat16, true>(WD, map, a, ss.nsq, st);
        case FDKOD_F16: return launch_tma_w<__half, true>(WD, map, a, ss.nsq, st);
    }
    return cudaErrorInvalidValue;
}

// dynamic shared memory of the pair kernel: kPairSlots slots of VPS views,
// two windows per view, plus the 128-byte alignment slack
inline size_t pair_smem(int es, int vps, int tile_stride) {
    return (size_t)es * kPairSlots * vps * 2 * tile_stride + 128;
}

template <typename TS, bool DIRECT, int WD, int VPS>
cudaError_t launch_pair_t(const CUtensorMap &map, const BpPairParams &prm, int nsq, cudaStream_t st) {
    const size_t smem = pair_smem((int)sizeof(TS), VPS, prm.tile_stride);
    cudaError_t e = ensure_smem<bp_pair_kernel<TS, DIRECT, WD, VPS>>(smem);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)(nsq * prm.tps * prm.tps), (unsigned)((prm.pend - prm.pbase + kZP - 1) / kZP));
    bp_pair_kernel<TS, DIRECT, WD, VPS><<<grid, kPairThreads, smem, st>>>(map, prm);
    return cudaGetLastError();
}

// views per slot: 2 (three CTAs per SM hold their ring at the usual window
// sizes), or 1 for larger windows (the staging depth only; the arithmetic and
// the result are the same)
template <typename TS, bool DIRECT, int WD>
cudaError_t launch_pair_v(int vps, const CUtensorMap &map, const BpPairParams &prm, int nsq, cudaStream_t st) {
    return vps == 2 ? launch_pair_t<TS, DIRECT, WD, 2>(map, prm, nsq, st)
                    : launch_pair_t<TS, DIRECT, WD, 1>(map, prm, nsq, st);
}

template <typename TS, bool DIRECT>
cudaError_t launch_pair_w(int WD, int vps, const CUtensorMap &map, const BpPairParams &prm, int nsq,
                          cudaStream_t st) {
    switch (WD) {
        case 32: return launch_pair_v<TS, DIRECT, 32>(vps, map, prm, nsq, st);
        case 48: return launch_pair_v<TS, DIRECT, 48>(vps, map, prm, nsq, st);
        case 64: return launch_pair_v<TS, DIRECT, 64>(vps, map, prm, nsq, st);
        case 96: return launch_pair_v<TS, DIRECT, 96>(vps, map, prm, nsq, st);
        case 128: return launch_pair_v<TS, DIRECT, 128>(vps, map, prm, nsq, st);
    }
    return cudaErrorInvalidValue;
}

// opt-in shared memory per block of the current device, less room for the
// kernels' static shared memory; *per_sm: the SM's shared memory less what
// the runtime reserves per block, shared by the CTAs of an SM
size_t smem_budget(size_t *per_sm = nullptr) {
    int dev = 0, optin = 0, sm = 0, reserved = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev) != cudaSuccess)
        return 0;
    if (per_sm) *per_sm = (size_t)sm;
    return optin > 2048 ? (size_t)optin - 2048 : 0;
}

// The mirrored-pair kernel serves launches over the whole detector and the
// slice pairs p0 .. p1 - 1 (slices p and N - 1 - p), with the TMA
// conditions of make_tma_launch and windows of kZP slices.
cudaError_t try_launch_pair(const PlanImpl &p, const SquareSet &ss, bool direct, const void *src, float *vol,
                            cudaStream_t st, int p0, int p1, bool &launched) {
    launched = false;
    const int es = (direct && p.qtype != FDKOD_F32) ? 2 : 4;
    const int WD = es == 4 ? ss.WdT : ss.WdT16;
    if (WD == 0 || ss.Rw2 > 256 || ((uintptr_t)src & 15) != 0) return cudaSuccess;
    if (direct && ((size_t)p.g.Nu * es) % 16 != 0) return cudaSuccess;
    uint64_t dims[3], strides[2];
    if (direct) {
        dims[0] = (uint64_t)p.g.Nu;
        dims[1] = (uint64_t)p.g.Nv;
        dims[2] = (uint64_t)p.g.P;
        strides[0] = (uint64_t)p.g.Nu * es;
    } else {
        dims[0] = (uint64_t)p.Tstride;
        dims[1] = (uint64_t)p.g.Nv;
        dims[2] = (uint64_t)ss.nsq * p.Pd;
        strides[0] = (uint64_t)p.Tstride * sizeof(float);
    }
    strides[1] = strides[0] * dims[1];
    const uint32_t box[3] = {(uint32_t)WD, (uint32_t)ss.Rw2, 1u};
    const CUtensorMapDataType dt = es == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                   : (p.qtype == FDKOD_F16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                                           : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16);
    CUtensorMap map;
    if (encode_map_3d(&map, dt, src, dims, strides, box) != cudaSuccess) return cudaSuccess;
    BpPairParams a{};
    a.vol = vol;
    a.geo = ss.geo;
    a.crop = ss.crop;
    a.w0 = ss.w0;
    a.status = p.status;
    a.N = p.g.N;
    a.P = p.g.P;
    a.Nv = p.g.Nv;
    a.m = ss.m;
    a.tps = ss.tiles_per_side;
    a.Pd = p.Pd;
    a.RW = ss.Rw2;
    a.tile_stride = (ss.Rw2 * WD + (128 / es - 1)) & ~(128 / es - 1);
    size_t per_sm = 0;
    const size_t budget = smem_budget(&per_sm);
    // 2 views per slot where three CTAs fit an SM (each with its static
    // shared memory and the runtime's reserve, 2 KiB together at most), else
    // 1 if one CTA fits
    const int vps = 3 * (pair_smem(es, 2, a.tile_stride) + 2048) <= per_sm ? 2
                    : (pair_smem(es, 1, a.tile_stride) <= budget ? 1 : 0);
    if (vps == 0) return cudaSuccess;  // windows too large: the 32-slice kernel
    a.pbase = p0;
    a.pend = p1;
    a.wait_ns = p.wait_ns > 0 ? (unsigned long long)p.wait_ns : kWaitLimitNs;
    a.fault = p.test_fault;
    if (direct) {
        a.nviews = p.g.P;
        a.vstep = 1;
        a.scale = (float)(M_PI / (double)p.g.P);
    } else {
        a.nviews = p.Pd;
        a.vstep = p.D;
        a.scale = (float)(M_PI / (double)p.Pd);
    }
    launched = true;
    if (!direct) return launch_pair_w<float, false>(WD, vps, map, a, ss.nsq, st);
    switch (p.qtype) {
        case FDKOD_F32: return launch_pair_w<float, true>(WD, vps, map, a, ss.nsq, st);
        case FDKOD_BF16: return launch_pair_w<__nv_bfloat16, true>(WD, vps, map, a, ss.nsq, st);
        case FDKOD_F16: return launch_pair_w<__half, true>(WD, vps, map, a, ss.nsq, st);
    }
    return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t launch_backproject_pairs(const PlanImpl &p, const SquareSet &ss, bool direct, const void *src,
                                     float *vol, cudaStream_t st, int p0, int p1, bool &launched) {
    return try_launch_pair(p, ss, direct, src, vol, st, p0, p1, launched);
}

cudaError_t launch_backproject(const PlanImpl &p, const SquareSet &ss, bool direct, const void *src, float *vol,
                               cudaStream_t st, Band b) {
    const bool whole = b.row0 == 0 && (b.nrows < 0 || b.nrows == p.g.Nv) && b.zoff == 0 && (b.nz < 0 || b.nz == p.g.N);
    if (b.nrows < 0) b.nrows = p.g.Nv;
    if (b.nz < 0) b.nz = p.g.N;
    bool launched = false;
    if (whole) {
        cudaError_t pe = try_launch_pair(p, ss, direct, src, vol, st, 0, (p.g.N + 1) / 2, launched);
        if (launched || pe != cudaSuccess) return pe;
    }
    cudaError_t te = try_launch_tma(p, ss, direct, src, vol, st, b, launched);
    if (launched || te != cudaSuccess) return te;
    BpParams a{};
    a.src = src;
    a.vol = vol;
    a.geo = ss.geo;
    a.crop = ss.crop;
    a.w0 = ss.w0;
    a.status = p.status;
    a.N = p.g.N;
    a.P = p.g.P;
    a.Nv = p.g.Nv;
    a.m = ss.m;
    a.tps = ss.tiles_per_side;
    a.Wd = ss.Wd;
    a.Rw = ss.Rw;
    const size_t per_view = sizeof(float) * (size_t)ss.Rw * (ss.Wd + 1);
    a.J = (int)std::min<size_t>(kViewsPerChunk, (200u * 1024u) / per_view);  // 0: the unstaged kernel
    a.row0 = b.row0;
    a.zoff = b.zoff;
    a.nz = b.nz;
    if (direct) {
        a.sq_stride = 0;
        a.view_stride = (long long)b.nrows * p.g.Nu;
        a.row_stride = p.g.Nu;
        a.src_cols = p.g.Nu;
        a.src_rows = b.nrows;
        a.nviews = p.g.P;
        a.vstep = 1;
        a.scale = (float)(M_PI / (double)p.g.P);
        switch (p.qtype) {
            case FDKOD_F32: return launch_t<float, true>(a, ss.nsq, st);
            case FDKOD_BF16: return launch_t<__nv_bfloat16, true>(a, ss.nsq, st);
            case FDKOD_F16: return launch_t<__half, true>(a, ss.nsq, st);
        }
        return cudaErrorInvalidValue;
    }
    a.view_stride = (long long)b.nrows * p.Tstride;
    a.sq_stride = (long long)p.Pd * a.view_stride;
    a.row_stride = p.Tstride;
    a.src_cols = p.Tstride;
    a.src_rows = b.nrows;
    a.nviews = p.Pd;
    a.vstep = p.D;
    a.scale = (float)(M_PI / (double)p.Pd);
    return launch_t<float, false>(a, ss.nsq, st);
}

// ---- batch of plans, one persistent launch --------------------------------

struct BatchImpl {
    CUtensorMap *maps = nullptr;
    BatchInst *insts = nullptr;
    int4 *items = nullptr;
    int *counter = nullptr;
    int nitems = 0;
    size_t smem = 0;
    int grid = 0;
};

namespace {
void batch_free_impl(BatchImpl *b) {
    cudaFree(b->maps);
    cudaFree(b->insts);
    cudaFree(b->items);
    cudaFree(b->counter);
    delete b;
}
}  // namespace

cudaError_t batch_create(const PlanImpl *const *plans, const void *const *src, float *const *vols, int count,
                         BatchImpl **out, bool &supported) {
    supported = false;
    *out = nullptr;
    std::vector<CUtensorMap> maps((size_t)count);
    std::vector<BatchInst> insts((size_t)count);
    std::vector<std::pair<double, int>> order;
    size_t smem = 0;
    for (int i = 0; i < count; ++i) {
        const PlanImpl &p = *plans[i];
        const bool direct = p.D == 1;
        if (direct && p.qtype != FDKOD_F32) return cudaSuccess;  // 16-bit windows: not in the batch form
        Band b;
        b.nrows = p.g.Nv;
        b.nz = p.g.N;
        int WD = 0;
        if (!make_tma_launch(p, p.od, direct, src[i], vols[i], b, maps[i], insts[i].a, WD)) return cudaSuccess;
        insts[i].a.wait_ns = kWaitLimitNs;  // the persistent form has no test hooks
        insts[i].a.fault = 0;
        insts[i].direct = direct ? 1 : 0;
        insts[i].WD = WD;
        smem = std::max(smem, sizeof(float) * (size_t)2 * kViewsPerStage * insts[i].a.tile_stride + 128);
        order.push_back({-(double)p.g.N * p.g.N * p.g.N * (double)insts[i].a.nviews, i});
    }
    std::sort(order.begin(), order.end());
    std::vector<int4> items;
    for (const auto &oi : order) {
        const int i = oi.second;
        const BpTmaParams &a = insts[i].a;
        const int tiles = plans[i]->od.nsq * a.tps * a.tps;
        const int zs = (a.nz + kZT - 1) / kZT;
        for (int t = 0; t < tiles; ++t)
            for (int z = 0; z < zs; ++z) items.push_back(make_int4(i, t, z, 0));
    }
    supported = true;
    cudaError_t e = ensure_smem<bp_persistent_kernel>(smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0, dev = 0, sms = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, bp_persistent_kernel, kThreads, smem)) !=
        cudaSuccess)
        return e;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    BatchImpl *b = new BatchImpl;
    b->nitems = (int)items.size();
    b->smem = smem;
    b->grid = std::min(per_sm * sms, std::max(1, b->nitems));
    if ((e = cudaMalloc(&b->maps, sizeof(CUtensorMap) * count)) != cudaSuccess ||
        (e = cudaMalloc(&b->insts, sizeof(BatchInst) * count)) != cudaSuccess ||
        (e = cudaMalloc(&b->items, sizeof(int4) * std::max<size_t>(1, items.size()))) != cudaSuccess ||
        (e = cudaMalloc(&b->counter, sizeof(int))) != cudaSuccess ||
        (e = cudaMemcpy(b->maps, maps.data(), sizeof(CUtensorMap) * count, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(b->insts, insts.data(), sizeof(BatchInst) * count, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(b->items, items.data(), sizeof(int4) * items.size(), cudaMemcpyHostToDevice)) !=
            cudaSuccess) {
        batch_free_impl(b);
        return e;
    }
    *out = b;
    return cudaSuccess;
}

cudaError_t batch_launch(const BatchImpl &b, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(b.counter, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    bp_persistent_kernel<<<b.grid, kThreads, b.smem, st>>>(b.maps, b.insts, b.items, b.nitems, b.counter);
    return cudaGetLastError();
}

void batch_destroy(BatchImpl *b) {
    if (b) batch_free_impl(b);
}

}  // namespace fdkod
