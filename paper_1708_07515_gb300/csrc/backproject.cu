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

#include "fdkod_internal.cuh"

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
bp_kernel(BpParams a) {
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
    const int z0 = blockIdx.y * kZT;
    const int z1 = min(z0 + kZT - 1, a.N - 1);

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
            const float gf = (float)ge.g;
            const float toff = DIRECT ? ge.frac - (float)w0q : -(float)w0q;
            const int c = lane & 7;
            const float cx = (float)((c & 1) ? xe : x0) - half_n - xc;
            const float cy = (float)((c & 2) ? ye : y0) - half_n - yc;
            const float cz = (float)((c & 4) ? z1 : z0) - half_n - zc;
            const float dd = fmaf(ge.cb, cx, ge.sb * cy);
            const float invU = gf / fmaf(ge.r, dd, 1.0f);
            const float t = fmaf(invU, fmaf(ge.alpha, cx, ge.gamma * cy), toff);
            const float zq = zc * ge.r * dd;
            const double vcen = fma((double)zc, ge.g, vcd);
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
            const int v = s_vlo[w] + r;
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
            if (z0 + i <= z1) a.vol[((size_t)(z0 + i) * a.N + y) * a.N + x] = acc[i] * a.scale;
    }
}

template <typename TS, bool DIRECT>
cudaError_t launch_t(BpParams prm, int nsq, cudaStream_t st) {
    const size_t smem = sizeof(float) * (size_t)prm.J * prm.Rw * (prm.Wd + 1);
    cudaError_t e = cudaFuncSetAttribute(bp_kernel<TS, DIRECT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)(nsq * prm.tps * prm.tps), (unsigned)((prm.N + kZT - 1) / kZT));
    bp_kernel<TS, DIRECT><<<grid, kThreads, smem, st>>>(prm);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_backproject(const PlanImpl &p, const SquareSet &ss, bool direct, const void *src, float *vol,
                               cudaStream_t st) {
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
    a.J = (int)std::min<size_t>(kViewsPerChunk, (200u * 1024u) / per_view);
    if (a.J < 1) return cudaErrorInvalidConfiguration;
    if (direct) {
        a.sq_stride = 0;
        a.view_stride = (long long)p.g.Nv * p.g.Nu;
        a.row_stride = p.g.Nu;
        a.src_cols = p.g.Nu;
        a.src_rows = p.g.Nv;
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
    a.view_stride = (long long)p.g.Nv * p.Tstride;
    a.sq_stride = (long long)p.Pd * a.view_stride;
    a.row_stride = p.Tstride;
    a.src_cols = p.Tstride;
    a.src_rows = p.g.Nv;
    a.nviews = p.Pd;
    a.vstep = p.D;
    a.scale = (float)(M_PI / (double)p.Pd);
    return launch_t<float, false>(a, ss.nsq, st);
}

}  // namespace fdkod
