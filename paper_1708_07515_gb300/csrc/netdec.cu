// Learned angular decimation (Sec. 2.1 leaves the low-pass of the
// decomposition open and says its implementation sets the quality).  The
// decimated view of square q is the plain low-pass plus a residual network
// along the view axis, applied to each shifted column (v, t) as an
// independent sequence x[k] = S_q[k][v][t] over the closed orbit:
//
//   a1[c][k] = relu(sum_m W1[c][m] x[k + m - 2])                 1 -> 16
//   a2[c][k] = relu(sum_{c', m} W2[c][c'][m] a1[c'][k + m - 2])  16 -> 16
//   S'[j]    = sum_{|i| < H D} h[|i|] x[j D + i]
//            + sum_{c, m} W3[c][m] a2[c][j D + m - 2]            16 -> 1, stride D
//
// Inference (net_decompose_kernel) keeps everything on chip: one CTA per
// (square, detector row, 16 shifted columns) walks the orbit in chunks of
// output views.  Two producer warps interpolate the shifted samples x of the
// next chunk from Q (FP32) into a double-buffered tile; eight consumer warps
// run the three layers as three rounds of tcgen05.mma on 8 tiles of 128
// operand rows, one row per (view, column), BF16 operands in shared memory
// (32-byte swizzle layout, tc5.cuh), FP32 accumulators in tensor memory:
// layer 1 against W1 with the 8 view taps of x as K (an im2col row), layer
// 2 as five MMAs per tile whose A operand starts 16 m rows (m views) further
// down -- the taps cost no data movement -- and layer 3 with its 5 taps as
// N.  Between rounds each thread reads its accumulator row (tcgen05.ld) and
// writes ReLU + BF16 in one conversion; the plain low-pass of the output
// views runs on the CUDA cores during the layer-1 round; the layer-3 terms
// go through shared memory and each output view sums its five.
//
// Training (CUDA cores, FP32): net_adjoint_kernel applies the adjoint of the
// backprojection to a residual volume (the gradient of the reconstruction
// error with respect to the decomposed data); net_backward_kernel recomputes
// the forward per chunk and back-propagates that gradient to the weights.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "fdkod_internal.cuh"
#include "tc5.cuh"
#include "tma.cuh"

namespace fdkod {
namespace {

constexpr int kC = kNetChannels, kK = kNetTaps;
constexpr int kG = 16;                 // shifted columns per CTA
constexpr int kTileViews = 128 / kG;   // views per 128-row MMA tile
constexpr int kTiles = 8;              // tiles per chunk
constexpr int kNA1 = kTiles * kTileViews;  // a1 views per chunk (a2 rows are computed for as many)
constexpr int kKA = kNA1 - 4;          // a2 views per chunk with their whole support
constexpr int kRowsA = kNA1 * kG + 64; // operand rows: the layer-2 taps read 64 rows past the tiles
constexpr int kRowBytes = 32;          // operand row: 16 BF16 values, 32-byte swizzle layout
constexpr int kOperandBytes = kRowsA * kRowBytes;
constexpr int kNetThreads = 256;
constexpr uint32_t kTmemCols = kTiles * 16;
constexpr uint64_t kNetWaitNs = 2000000000ull;

__device__ __forceinline__ float ld_q(const float *p) { return __ldg(p); }
__device__ __forceinline__ float ld_q(const __nv_bfloat16 *p) { return __bfloat162float(__ldg(p)); }
__device__ __forceinline__ float ld_q(const __half *p) { return __half2float(__ldg(p)); }

__device__ __forceinline__ int wrap(int k, int P) {
    k %= P;
    return k < 0 ? k + P : k;
}

// shifted sample x of view k, column t of square q on row `row` (zero past
// the square's row length T and outside the detector): the interpolation of
// the plain decomposition
template <typename TQ>
__device__ __forceinline__ float shifted_sample(const TQ *__restrict__ Q, const int32_t *__restrict__ crop,
                                                const GeomEntry *__restrict__ geo, int q, int k, int t, int T,
                                                int row, int nrows, int P, int Nu) {
    if (t >= T) return 0.f;
    const size_t o = (size_t)q * P + k;
    const int c = __ldg(crop + o) + t;
    const float f = __ldg(&geo[o].frac);
    const TQ *r = Q + ((size_t)k * nrows + row) * Nu;
    const float a = (c >= 0 && c < Nu) ? ld_q(r + c) : 0.f;
    const float b = (c + 1 >= 0 && c + 1 < Nu) ? ld_q(r + c + 1) : 0.f;
    return fmaf(f, b - a, a);
}

// two floats -> BF16 pair (lo in the low half), negative values to 0
__device__ __forceinline__ uint32_t relu_bf16x2(float lo, float hi) {
    uint32_t r;
    asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
    return r;
}
__device__ __forceinline__ uint32_t bf16x2(float lo, float hi) {
    const __nv_bfloat162 b = __floats2bfloat162_rn(lo, hi);
    return *(const uint32_t *)&b;
}

struct NetChunk {
    int J;    // output views per chunk
    int XL;   // x views before the chunk's first output view
    int NX;   // x views per chunk
};

__host__ __device__ inline NetChunk net_chunk(int D, int HD) {
    NetChunk c;
    c.J = (kKA - 5) / D + 1;
    c.XL = HD - 1 > 6 ? HD - 1 : 6;
    const int a = kNA1 + c.XL + 1, b = (c.J - 1) * D + HD + c.XL;
    c.NX = a > b ? a : b;
    return c;
}

// dynamic shared memory of net_decompose_kernel (bytes, after 128-byte alignment)
__host__ __device__ inline size_t net_smem(const NetChunk &c, int HD) {
    return (size_t)kOperandBytes + sizeof(uint16_t) * (kK + 2) * 256 + 2 * sizeof(float) * (size_t)c.NX * kG +
           sizeof(float) * (size_t)c.J * kG + sizeof(float) * (size_t)HD;
}

// barrier 1: the consumer warps only (the producers run ahead)
__device__ __forceinline__ void consumers_sync() { asm volatile("bar.sync 1, %0;" ::"n"(kNetThreads) : "memory"); }
__device__ __forceinline__ bool consumers_and(bool v) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 p, %1, 0;\n\t"
        "bar.red.and.pred q, 1, %2, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)v), "n"(kNetThreads)
        : "memory");
    return r != 0;
}

// One CTA per (square q, detector row v, 16 shifted columns); the orbit is
// walked in chunks of J output views.  Two producer warps interpolate the
// shifted samples x of the next chunk into the other half of a
// double-buffered tile (mbarriers full / empty) while eight consumer warps
// work on the current one.  Per chunk the consumers run (operand rows are
// (view, column) pairs, row = view * 16 + column; three rounds on the
// tensor cores, M = 128 rows x N = 16 per tile, 8 tiles, FP32 in tensor
// memory, BF16 operands in shared memory):
//   1. layer-1 operand: row (view, column) = x at views view - 2 .. view + 5
//      (BF16; taps 5..7, and the row's second 16 bytes, meet zero weights)
//   2. z1 = one MMA per tile against W1 (K = 16 taps); meanwhile the plain
//      low-pass of the chunk's output views (FP32, from x)
//   3. a1 = relu(z1) as BF16, one 32-byte row of 16 channels per operand row
//   4. z2 = five MMAs per tile, tap m reading a1 from row 16 m on (K = 16 channels)
//   5. a2 = relu(z2) as BF16, over a1
//   6. p = one MMA per tile against W3 (N = its 5 taps, zero-padded)
//   7. each row's p[0..4] to shared memory
//   8. output view = plain low-pass + the five p[m] of the rows it reads; store
constexpr int kProducerWarps = 2;
constexpr int kNetCtaThreads = kNetThreads + 32 * kProducerWarps;

template <typename TQ>
__global__ void __launch_bounds__(kNetCtaThreads, 4)
net_decompose_kernel(const TQ *__restrict__ Q, float *__restrict__ out, const int32_t *__restrict__ crop,
                     const GeomEntry *__restrict__ geo, const int32_t *__restrict__ Tq,
                     const NetWeights *__restrict__ net, int *status, int Tstride, int P, int D, int Pd, int HD,
                     int nrows, int Nu, int ngroups) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    // 1024-byte aligned (the swizzle pattern repeats every 256 bytes)
    unsigned char *base = smem_raw + ((1024u - (tma::smem_u32(smem_raw) & 1023u)) & 1023u);
    __shared__ __align__(8) uint64_t bar, full[2], empty[2];
    __shared__ uint32_t tmem_slot;

    const int q = blockIdx.x / ngroups, grp = blockIdx.x - q * ngroups;
    const int v = blockIdx.y;
    const int t0 = grp * kG;
    const int T = __ldg(Tq + q);
    const size_t jstride = (size_t)nrows * Tstride;
    float *outq = out + ((size_t)q * Pd * nrows + v) * Tstride;
    const int tid = threadIdx.x;
    if (t0 >= T) {  // past this square's row length: zeros (uniform per CTA)
        for (int i = tid; i < Pd * kG; i += kNetCtaThreads) {
            const int j = i / kG, t = t0 + i % kG;
            if (t < Tstride) outq[(size_t)j * jstride + t] = 0.f;
        }
        return;
    }
    const NetChunk ch = net_chunk(D, HD);
    unsigned char *opa = base;                                      // operands: kRowsA rows of 32 bytes
    unsigned char *wb = opa + kOperandBytes;                        // W2 (5 x 512 B), W1 (512 B), W3 (512 B)
    float *xbuf = (float *)(wb + sizeof(uint16_t) * (kK + 2) * 256);  // 2 x [NX][kG]
    float *yacc = xbuf + 2 * (size_t)ch.NX * kG;                    // [J][kG]
    float *hs = yacc + (size_t)ch.J * kG;                           // [HD]

    for (int i = tid; i < (kK + 2) * 256 / 8; i += kNetCtaThreads)
        ((uint4 *)wb)[i] = ((const uint4 *)net->w2)[i];  // w2, b1, b3 are contiguous
    for (int i = tid; i < HD; i += kNetCtaThreads) hs[i] = net->h[i];
    // rows past the tiles: read by the tap offsets, must hold finite values
    for (int i = tid; i < 2 * 64; i += kNetCtaThreads)
        *(uint4 *)(opa + (size_t)(kNA1 * kG) * kRowBytes + (size_t)i * 16) = make_uint4(0u, 0u, 0u, 0u);
    if (tid == 0) {
        tma::mbar_init(&bar, 1);
        for (int b = 0; b < 2; ++b) {
            tma::mbar_init(&full[b], 32 * kProducerWarps);
            tma::mbar_init(&empty[b], kNetThreads);
        }
        tma::fence_mbar_init();
    }
    if (tid < 32) tc5::alloc(&tmem_slot, kTmemCols);
    tc5::fence_before_sync();
    __syncthreads();
    tc5::fence_after_sync();
    const uint32_t tmem = tmem_slot;
    const int warp = tid >> 5, lane = tid & 31;
    const int nchunks = (Pd + ch.J - 1) / ch.J;

    if (warp >= kNetThreads / 32) {
        // ---- producers: x of chunk cc into buffer cc % 2; thread pt covers
        // column g = pt % 16 of views pt / 16, + 4, + 8, ...
        const int pt = tid - kNetThreads, g = pt & (kG - 1);
        const size_t qo = (size_t)q * P;
        const TQ *Qv = Q + (size_t)v * Nu;
        const size_t view_stride = (size_t)nrows * Nu;
        const bool col_in = t0 + g < T;
        for (int cc = 0; cc < nchunks; ++cc) {
            const int b = cc & 1;
            if (cc >= 2 && !tma::mbar_wait_bounded(&empty[b], (uint32_t)(((cc >> 1) - 1) & 1), kNetWaitNs)) {
                atomicOr(status, 2);
                break;
            }
            float *xs = xbuf + (size_t)b * ch.NX * kG;
            int k = cc * ch.J * D - ch.XL + (pt >> 4);
            if (k < 0 || k >= P) k = wrap(k, P);
#pragma unroll 8
            for (int ix = pt >> 4; ix < ch.NX; ix += 32 * kProducerWarps / kG) {
                const size_t o = qo + k;
                const int c = __ldg(crop + o) + t0 + g;
                const float f = __ldg(&geo[o].frac);
                const TQ *r = Qv + (size_t)k * view_stride;
                const float a = (col_in && c >= 0 && c < Nu) ? ld_q(r + c) : 0.f;
                const float bb = (col_in && c + 1 >= 0 && c + 1 < Nu) ? ld_q(r + c + 1) : 0.f;
                xs[ix * kG + g] = fmaf(f, bb - a, a);
                k += 32 * kProducerWarps / kG;
                if (k >= P) k = wrap(k, P);
            }
            tma::mbar_arrive(&full[b]);
        }
    } else {
        // ---- consumers
        const int wq = warp & 3, wh = warp >> 2;  // tensor-memory lane quarter, half of the tiles
        const uint32_t sopa = tma::smem_u32(opa), swb = tma::smem_u32(wb);
        constexpr uint32_t kIdesc = tc5::idesc_bf16_f32(128, 16);
        // descriptors: operands in the 32-byte swizzle layout (a row = 16
        // values; a tile = 128 rows = 256 units of 16 bytes, a view = 16 rows
        // = 32 units), weights unswizzled (two 256-byte planes)
        const uint64_t dA12 = tc5::smem_desc_sw32(sopa, 256);
        const uint64_t dX = dA12;
        const uint64_t dW2 = tc5::smem_desc(swb, 256, 128);
        const uint64_t dW1 = tc5::smem_desc(swb + kK * 512, 256, 128);
        const uint64_t dW3 = tc5::smem_desc(swb + (kK + 1) * 512, 256, 128);
        uint32_t phase = 0;
        bool failed = false;

        // wait for the MMAs committed last: one thread polls, the others
        // sleep in the barrier; false on timeout (uniform)
        auto mma_done = [&]() -> bool {
            const bool ok = tid != 0 || tma::mbar_wait_spin(&bar, phase, kNetWaitNs);
            phase ^= 1u;
            const bool all = consumers_and(ok);
            tc5::fence_after_sync();
            return all;
        };
        // after writing an operand: visible to the tensor cores, tensor-memory
        // reads of this thread ordered before the next MMA
        auto operands_ready = [&]() {
            tma::fence_proxy_async();
            tc5::fence_before_sync();
            consumers_sync();
            tc5::fence_after_sync();
        };
        // relu of tensor-memory rows -> BF16 operand rows; warp w reads
        // lanes 32 (w % 4) .. + 31 of tiles 4 (w / 4) .. + 3
        auto relu_to_operand = [&]() {
#pragma unroll 1
            for (int i = wh * (kTiles / 2); i < (wh + 1) * (kTiles / 2); ++i) {
                float z[16];
                tc5::ld16(tmem + ((uint32_t)(32 * wq) << 16) + (uint32_t)(16 * i), z);
                const int r = 128 * i + 32 * wq + lane;
                unsigned char *row = opa + (size_t)r * kRowBytes;
                const int sw = (r >> 2) & 1;  // 16-byte halves swapped in rows 4-7 of each group of 8
                *(uint4 *)(row + 16 * sw) = make_uint4(relu_bf16x2(z[0], z[1]), relu_bf16x2(z[2], z[3]),
                                                       relu_bf16x2(z[4], z[5]), relu_bf16x2(z[6], z[7]));
                *(uint4 *)(row + 16 * (sw ^ 1)) =
                    make_uint4(relu_bf16x2(z[8], z[9]), relu_bf16x2(z[10], z[11]), relu_bf16x2(z[12], z[13]),
                               relu_bf16x2(z[14], z[15]));
            }
        };

        for (int cc = 0; cc < nchunks && !failed; ++cc) {
            const int j0 = cc * ch.J;
            const int Jc = min(ch.J, Pd - j0);
            const int b = cc & 1;
            const float *xs = xbuf + (size_t)b * ch.NX * kG;
            const bool xok = tid != 0 || tma::mbar_wait_spin(&full[b], (uint32_t)((cc >> 1) & 1), kNetWaitNs);
            if (!consumers_and(xok)) {
                failed = true;
                break;
            }
            // 1. layer-1 operand: a1 view ka (= view j0 D - 4 + ka) reads x at
            // index ka + XL - 6 + t, t < 8; thread: column g, kVPT consecutive views
            {
                constexpr int kVPT = kNA1 * kG / kNetThreads;
                const int g = tid & (kG - 1), b4 = (tid >> 4) * kVPT;
                const float *xp = xs + (size_t)(b4 + ch.XL - 6) * kG + g;
                float xw[kVPT + 7];
#pragma unroll
                for (int t = 0; t < kVPT + 7; ++t) xw[t] = xp[t * kG];
#pragma unroll
                for (int i = 0; i < kVPT; ++i) {
                    const int r = (b4 + i) * kG + g;
                    unsigned char *row = opa + (size_t)r * kRowBytes;
                    const int sw = (r >> 2) & 1;
                    *(uint4 *)(row + 16 * sw) =
                        make_uint4(bf16x2(xw[i], xw[i + 1]), bf16x2(xw[i + 2], xw[i + 3]),
                                   bf16x2(xw[i + 4], xw[i + 5]), bf16x2(xw[i + 6], xw[i + 7]));
                    *(uint4 *)(row + 16 * (sw ^ 1)) = make_uint4(0u, 0u, 0u, 0u);  // taps 8-15: zero weights
                }
            }
            operands_ready();
            // 2. z1
            if (tid == 0) {
#pragma unroll 1
                for (int i = 0; i < kTiles; ++i)
                    tc5::mma_bf16(tmem + (uint32_t)(16 * i), dX + (uint64_t)(256 * i), dW1, kIdesc, 0u);
                tc5::commit(&bar);
            }
            // plain low-pass meanwhile: output view j0 + jl, column g; then x
            // is no longer needed: hand the buffer back to the producers
            for (int i = tid; i < Jc * kG; i += kNetThreads) {
                const int jl = i / kG, g = i - jl * kG;
                const float *xp = xs + (size_t)(jl * D + ch.XL) * kG + g;
                float acc = hs[0] * xp[0];
                for (int d = 1; d < HD; ++d) acc = fmaf(hs[d], xp[(size_t)d * kG] + xp[-(ptrdiff_t)d * kG], acc);
                yacc[i] = acc;
            }
            tma::mbar_arrive(&empty[b]);
            if (!mma_done()) {
                failed = true;
                break;
            }
            // 3. a1
            relu_to_operand();
            operands_ready();
            // 4. z2: tile i = a2 views 8 i .. 8 i + 7 (view ka2 = view j0 D - 2
            // + ka2); tap m reads a1 from row 16 m on
            if (tid == 0) {
                // tap-major order: consecutive MMAs write different tiles
#pragma unroll
                for (int m = 0; m < kK; ++m)
#pragma unroll 1
                    for (int i = 0; i < kTiles; ++i)
                        tc5::mma_bf16(tmem + (uint32_t)(16 * i), dA12 + (uint64_t)(256 * i + 32 * m),
                                      dW2 + (uint64_t)(32 * m), kIdesc, m > 0 ? 1u : 0u);
                tc5::commit(&bar);
            }
            if (!mma_done()) {
                failed = true;
                break;
            }
            // 5. a2
            relu_to_operand();
            operands_ready();
            // 6. layer-3 terms p[row][m] = sum_c W3[c][m] a2[row][c]
            if (tid == 0) {
#pragma unroll 1
                for (int i = 0; i < kTiles; ++i)
                    tc5::mma_bf16(tmem + (uint32_t)(16 * i), dA12 + (uint64_t)(256 * i), dW3, kIdesc, 0u);
                tc5::commit(&bar);
            }
            if (!mma_done()) {
                failed = true;
                break;
            }
            // 7. the layer-3 terms of every row to shared memory (over a2,
            // whose MMAs are done): pm[ka2][m][g], m < 5
            float *pm = (float *)opa;
#pragma unroll 1
            for (int i = wh * (kTiles / 2); i < (wh + 1) * (kTiles / 2); ++i) {
                float pz[8];  // taps 0..4 (columns 5..15 are the zero-padded N)
                tc5::ld8(tmem + ((uint32_t)(32 * wq) << 16) + (uint32_t)(16 * i), pz);
                const int ka2 = kTileViews * i + 2 * wq + (lane >> 4), g = lane & (kG - 1);
                float *dst = pm + (size_t)ka2 * kK * kG + g;
#pragma unroll
                for (int m = 0; m < kK; ++m) dst[m * kG] = pz[m];
            }
            tc5::fence_before_sync();
            consumers_sync();
            // 8. output view j0 + jl = plain low-pass + sum_m pm[jl D + m][m]
            for (int i = tid; i < Jc * kG; i += kNetThreads) {
                const int jl = i / kG, g = i - jl * kG, t = t0 + g;
                const float *src = pm + (size_t)jl * D * kK * kG + g;
                float y = yacc[i];
#pragma unroll
                for (int m = 0; m < kK; ++m) y += src[(size_t)(m * kK + m) * kG];
                if (t < Tstride) outq[(size_t)(j0 + jl) * jstride + t] = y;
            }
            // (the next chunk writes its layer-1 operand over pm only after
            // the barrier of its x wait)
        }
        if (failed && tid == 0) {
            // a wait gave up: report; if MMAs are in flight, give them
            // another bounded wait before tensor memory is freed
            atomicOr(status, 2);
            tma::mbar_wait_bounded(&bar, phase ^ 1u, kNetWaitNs);
        }
    }
    tc5::fence_before_sync();
    __syncthreads();
    tc5::fence_after_sync();
    if (tid < 32) tc5::dealloc(tmem, kTmemCols);
}

template <typename TQ>
cudaError_t launch_net_t(const PlanImpl &p, const TQ *Q, float *out, cudaStream_t st, int nrows) {
    const int HD = p.tap_blocks * p.D;
    const NetChunk ch = net_chunk(p.D, HD);
    const size_t smem = net_smem(ch, HD) + 1024;
    cudaError_t e = ensure_smem<net_decompose_kernel<TQ>>(smem);
    if (e != cudaSuccess) return e;
    const int ngroups = (p.Tstride + kG - 1) / kG;
    dim3 grid((unsigned)(ngroups * p.od.nsq), (unsigned)nrows);
    net_decompose_kernel<TQ><<<grid, kNetCtaThreads, smem, st>>>(Q, out, p.od.crop, p.od.geo, p.od.T, p.net, p.status,
                                                             p.Tstride, p.g.P, p.D, p.Pd, HD, nrows, p.g.Nu,
                                                             ngroups);
    return cudaGetLastError();
}


// ---------------------------------------------------------------------------
// Training kernels (FP32 on the CUDA cores).

// Adjoint of the backprojection of decomposed data, one slice: for every
// voxel (x, y) of slice z, e = vol - ref, and each decimated view j of the
// voxel's square q adds (pi / P') U^-2 e times the bilinear weight of the
// sample position the backprojection reads to dS[q][j][v][t] (t < T_q, v a
// row of the plan).  sq_err accumulates sum e^2.  The sample position is the
// backprojection's: 1/U = g / (1 + r (cb dx + sb dy)),
// t = (1/U)(alpha dx + gamma dy) - w0, v = z / U + (Nv - 1) / 2.
__global__ void __launch_bounds__(256)
net_adjoint_kernel(const float *__restrict__ vol, const float *__restrict__ ref, int z, float *__restrict__ dS,
                   float *sq_err, const GeomEntry *__restrict__ geo, const int32_t *__restrict__ w0,
                   const int32_t *__restrict__ Tq, int N, int s, int P, int D, int Pd, int Nv, int Tstride,
                   float scale) {
    const int ix = blockIdx.x * 16 + (threadIdx.x & 15), iy = blockIdx.y * 16 + (threadIdx.x >> 4);
    const bool in = ix < N && iy < N;
    const float e = in ? vol[(size_t)iy * N + ix] - ref[(size_t)iy * N + ix] : 0.f;
    float e2 = e * e;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) e2 += __shfl_xor_sync(0xffffffffu, e2, o);
    if ((threadIdx.x & 31) == 0 && e2 != 0.f) atomicAdd(sq_err, e2);
    if (!in || e == 0.f) return;
    const int m = 1 << s;
    const int qx = (int)(((int64_t)ix << s) / N), qy = (int)(((int64_t)iy << s) / N);
    const int q = qy * m + qx;
    auto first = [&](int c) { return (int)(((int64_t)c * N + m - 1) / m); };
    const float half_n = 0.5f * (float)(N - 1);
    const float xc = 0.5f * ((float)first(qx) + (float)(first(qx + 1) - 1)) - half_n;
    const float yc = 0.5f * ((float)first(qy) + (float)(first(qy + 1) - 1)) - half_n;
    const float dx = (float)ix - half_n - xc, dy = (float)iy - half_n - yc;
    const float zc = (float)z - half_n, vcd = 0.5f * (float)(Nv - 1);
    const int T = Tq[q];
    const float toff = -(float)w0[q];
    const size_t qo = (size_t)q * Pd * Nv * Tstride;
    for (int j = 0; j < Pd; ++j) {
        const GeomEntry ge = geo[(size_t)q * P + (size_t)j * D];
        const float dd = fmaf(ge.cb, dx, ge.sb * dy);
        const float invU = (ge.g_hi + ge.g_lo) / fmaf(ge.r, dd, 1.0f);
        const float t = fmaf(invU, fmaf(ge.alpha, dx, ge.gamma * dy), toff);
        const float v = fmaf(zc, invU, vcd);
        const float tf = floorf(t), vf = floorf(v);
        const float ft = t - tf, fv = v - vf;
        const int c0 = (int)tf, r0 = (int)vf;
        const float w = scale * invU * invU * e;
        float *row = dS + qo + (size_t)j * Nv * Tstride;
#pragma unroll
        for (int dr = 0; dr < 2; ++dr) {
            const int r = r0 + dr;
            if (r < 0 || r >= Nv) continue;
            const float wr = dr ? fv : 1.f - fv;
#pragma unroll
            for (int dc = 0; dc < 2; ++dc) {
                const int c = c0 + dc;
                if (c < 0 || c >= T) continue;
                atomicAdd(row + (size_t)r * Tstride + c, w * wr * (dc ? ft : 1.f - ft));
            }
        }
    }
}

// Backward pass of the net for one (square, detector row, 8 columns) and
// every output view, chunk by chunk (the chunking of the forward): recompute
// x, a1, a2 in FP32 with the FP32 weights w, take dS[q][j][v][t] as the
// gradient of the decimated views, and accumulate the weight gradient
// (layout of the C interface) into dW.  The plain low-pass has no weights.
constexpr int kBG = 8;                         // columns per CTA
constexpr int kBThreads = 256;
constexpr int kBA1 = kNA1 * kBG + 1;           // channel stride of a1 (padded)
constexpr int kBA2 = kKA * kBG + 1;            // channel stride of a2
__host__ __device__ inline size_t net_bwd_smem(const NetChunk &c) {
    return sizeof(float) * ((size_t)kNetSize + (size_t)c.NX * kBG + (size_t)c.J * kBG + (size_t)kC * kBA1 +
                            (size_t)kC * kBA2);
}

template <typename TQ>
__global__ void __launch_bounds__(kBThreads)
net_backward_kernel(const TQ *__restrict__ Q, const float *__restrict__ wts, const float *__restrict__ dS,
                    float *__restrict__ dW, const int32_t *__restrict__ crop, const GeomEntry *__restrict__ geo,
                    const int32_t *__restrict__ Tq, int Tstride, int P, int D, int Pd, int HD, int Nv, int Nu,
                    int ngroups, int row_lo) {
    extern __shared__ __align__(16) float fsm[];
    const NetChunk ch = net_chunk(D, HD);
    float *W = fsm;                                  // W1 [80] W2 [1280] W3 [80]
    float *xs = W + kNetSize;                        // [NX][kBG]
    float *dy = xs + (size_t)ch.NX * kBG;            // [J][kBG]
    float *a1 = dy + (size_t)ch.J * kBG;             // [kC][kBA1]: a1, then dz1
    float *a2 = a1 + (size_t)kC * kBA1;              // [kC][kBA2]: a2, then dz2
    const float *W1 = W, *W2 = W + kC * kK, *W3 = W + kC * kK + kC * kC * kK;
    const int q = blockIdx.x / ngroups, grp = blockIdx.x - q * ngroups;
    const int v = row_lo + blockIdx.y;
    const int t0 = grp * kBG;
    const int T = Tq[q];
    if (t0 >= T) return;
    const int tid = threadIdx.x;
    for (int i = tid; i < kNetSize; i += kBThreads) W[i] = wts[i];
    float g1 = 0.f, g3 = 0.f, g2[kK] = {0.f, 0.f, 0.f, 0.f, 0.f};
    const int cw = tid >> 4, cv = tid & 15;        // (c, c') of this thread's W2 gradients
    const int nchunks = (Pd + ch.J - 1) / ch.J;
    __syncthreads();
    for (int cc = 0; cc < nchunks; ++cc) {
        const int j0 = cc * ch.J, Jc = min(ch.J, Pd - j0);
        const int kx0 = j0 * D - ch.XL;
        for (int i = tid; i < ch.NX * kBG; i += kBThreads) {
            const int ix = i / kBG, g = i - ix * kBG;
            xs[i] = shifted_sample(Q, crop, geo, q, wrap(kx0 + ix, P), t0 + g, T, v, Nv, P, Nu);
        }
        for (int i = tid; i < ch.J * kBG; i += kBThreads) {
            const int jl = i / kBG, t = t0 + (i - jl * kBG);
            dy[i] = (jl < Jc && t < T) ? dS[(((size_t)q * Pd + j0 + jl) * Nv + v) * Tstride + t] : 0.f;
        }
        __syncthreads();
        // layer 1 (a1 view ka = view j0 D - 4 + ka)
        for (int i = tid; i < kC * kNA1 * kBG; i += kBThreads) {
            const int c = i / (kNA1 * kBG), p = i - c * (kNA1 * kBG);
            const float *xp = xs + (size_t)(p / kBG + ch.XL - 6) * kBG + (p % kBG);
            float z = 0.f;
#pragma unroll
            for (int m = 0; m < kK; ++m) z = fmaf(W1[c * kK + m], xp[m * kBG], z);
            a1[c * kBA1 + p] = fmaxf(z, 0.f);
        }
        __syncthreads();
        // layer 2 (a2 view ka2 = view j0 D - 2 + ka2 reads a1 views ka2 .. ka2 + 4)
        for (int i = tid; i < kC * kKA * kBG; i += kBThreads) {
            const int c = i / (kKA * kBG), p = i - c * (kKA * kBG);
            float z = 0.f;
            for (int ci = 0; ci < kC; ++ci) {
                const float *w = W2 + (c * kC + ci) * kK;
                const float *ap = a1 + ci * kBA1 + p;
#pragma unroll
                for (int m = 0; m < kK; ++m) z = fmaf(w[m], ap[m * kBG], z);
            }
            a2[c * kBA2 + p] = fmaxf(z, 0.f);
        }
        __syncthreads();
        // layer 3 weights: dW3[c][m] = sum_{jl, g} dy[jl][g] a2[c][jl D + m][g]
        if (tid < kC * kK) {
            const int c = tid / kK, m = tid - c * kK;
            for (int jl = 0; jl < Jc; ++jl)
                for (int g = 0; g < kBG; ++g) g3 = fmaf(dy[jl * kBG + g], a2[c * kBA2 + (jl * D + m) * kBG + g], g3);
        }
        __syncthreads();
        // dz2 in place of a2: relu'(z2) sum_jl W3[c][ka2 - jl D] dy[jl]
        for (int i = tid; i < kC * kKA * kBG; i += kBThreads) {
            const int c = i / (kKA * kBG), p = i - c * (kKA * kBG);
            const int ka2 = p / kBG, g = p - ka2 * kBG;
            float d = 0.f;
            if (a2[c * kBA2 + p] > 0.f) {
                int jl = ka2 >= 4 ? (ka2 - 4 + D - 1) / D : 0;
                for (; jl * D <= ka2 && jl < Jc; ++jl) d = fmaf(W3[c * kK + ka2 - jl * D], dy[jl * kBG + g], d);
            }
            a2[c * kBA2 + p] = d;
        }
        __syncthreads();
        // layer 2 weights: dW2[cw][cv][m] = sum_p dz2[cw][p] a1[cv][p + m kBG]
        {
            const float *dz = a2 + cw * kBA2;
            const float *ap = a1 + cv * kBA1;
            for (int p = 0; p < kKA * kBG; ++p) {
                const float d = dz[p];
#pragma unroll
                for (int m = 0; m < kK; ++m) g2[m] = fmaf(d, ap[p + m * kBG], g2[m]);
            }
        }
        __syncthreads();
        // dz1 in place of a1: relu'(z1) sum_{c, m} W2[c][c'][m] dz2[c][ka - m]
        for (int i = tid; i < kC * kNA1 * kBG; i += kBThreads) {
            const int ci = i / (kNA1 * kBG), p = i - ci * (kNA1 * kBG);
            const int ka = p / kBG, g = p - ka * kBG;
            float d = 0.f;
            if (a1[ci * kBA1 + p] > 0.f) {
                for (int c = 0; c < kC; ++c) {
                    const float *w = W2 + (c * kC + ci) * kK;
                    const float *dz = a2 + c * kBA2 + g;
#pragma unroll
                    for (int m = 0; m < kK; ++m) {
                        const int k2 = ka - m;
                        if (k2 >= 0 && k2 < kKA) d = fmaf(w[m], dz[k2 * kBG], d);
                    }
                }
            }
            a1[ci * kBA1 + p] = d;
        }
        __syncthreads();
        // layer 1 weights: dW1[c][m] = sum_p dz1[c][p] x[p + m]
        if (tid < kC * kK) {
            const int c = tid / kK, m = tid - c * kK;
            for (int p = 0; p < kNA1 * kBG; ++p)
                g1 = fmaf(a1[c * kBA1 + p], xs[(size_t)(p / kBG + ch.XL - 6 + m) * kBG + (p % kBG)], g1);
        }
        __syncthreads();
    }
    if (tid < kC * kK) {
        atomicAdd(dW + tid, g1);
        atomicAdd(dW + kC * kK + kC * kC * kK + tid, g3);
    }
#pragma unroll
    for (int m = 0; m < kK; ++m) atomicAdd(dW + kC * kK + (cw * kC + cv) * kK + m, g2[m]);
}

template <typename TQ>
cudaError_t launch_backward_t(const PlanImpl &p, const TQ *Q, const float *w, const float *dS, int row_lo,
                              int row_hi, float *dW, cudaStream_t st) {
    const int HD = p.tap_blocks * p.D;
    const NetChunk ch = net_chunk(p.D, HD);
    const size_t smem = net_bwd_smem(ch);
    cudaError_t e = ensure_smem<net_backward_kernel<TQ>>(smem);
    if (e != cudaSuccess) return e;
    const int ngroups = (p.Tstride + kBG - 1) / kBG;
    dim3 grid((unsigned)(ngroups * p.od.nsq), (unsigned)(row_hi - row_lo));
    net_backward_kernel<TQ><<<grid, kBThreads, smem, st>>>(Q, w, dS, dW, p.od.crop, p.od.geo, p.od.T, p.Tstride,
                                                          p.g.P, p.D, p.Pd, HD, p.g.Nv, p.g.Nu, ngroups, row_lo);
    return cudaGetLastError();
}

// round to the nearest BF16, ties to even (finite inputs)
uint16_t bf16_bits(float f) {
    uint32_t u;
    std::memcpy(&u, &f, 4);
    u += 0x7FFFu + ((u >> 16) & 1u);
    return (uint16_t)(u >> 16);
}
float bf16_value(uint16_t b) {
    const uint32_t u = (uint32_t)b << 16;
    float f;
    std::memcpy(&f, &u, 4);
    return f;
}

int net_status(cudaError_t e) {
    if (e == cudaSuccess) return FDKOD_OK;
    return e == cudaErrorMemoryAllocation ? FDKOD_ERR_OOM : FDKOD_ERR_CUDA;
}

}  // namespace

cudaError_t launch_net_decompose(const PlanImpl &p, const void *Q, float *out, cudaStream_t st, int nrows) {
    switch (p.qtype) {
        case FDKOD_F32: return launch_net_t(p, (const float *)Q, out, st, nrows);
        case FDKOD_BF16: return launch_net_t(p, (const __nv_bfloat16 *)Q, out, st, nrows);
        case FDKOD_F16: return launch_net_t(p, (const __half *)Q, out, st, nrows);
    }
    return cudaErrorInvalidValue;
}

cudaError_t upload_net(PlanImpl &p) {
    NetWeights h{};
    const float *W1 = p.net_host, *W2 = p.net_host + kC * kK, *W3 = W2 + kC * kC * kK;
    // B operands, N x K = 16 x 16, K-major: element (n, k) at uint16 index
    // (k / 8) 128 + n 8 + k % 8 (two 8-value planes of 256 bytes)
    auto at = [](int n, int k) { return (k / 8) * 128 + n * 8 + (k % 8); };
    for (int m = 0; m < kK; ++m)  // layer 2, tap m: n = output channel, k = input channel
        for (int c = 0; c < kC; ++c)
            for (int ci = 0; ci < kC; ++ci) h.w2[m * 256 + at(c, ci)] = bf16_bits(W2[(c * kC + ci) * kK + m]);
    for (int c = 0; c < kC; ++c)      // layer 1: n = channel, k = tap (taps 5..15 zero)
        for (int m = 0; m < kK; ++m) h.b1[at(c, m)] = bf16_bits(W1[c * kK + m]);
    for (int m = 0; m < kK; ++m)      // layer 3: n = tap (5..15 zero), k = channel
        for (int c = 0; c < kC; ++c) h.b3[at(m, c)] = bf16_bits(W3[c * kK + m]);
    for (int i = 0; i < 2 * kMaxTapD; ++i) h.h[i] = (float)p.htaps[i];
    return cudaMemcpy(p.net, &h, sizeof(h), cudaMemcpyHostToDevice);
}

}  // namespace fdkod

using fdkod::PlanImpl;

extern "C" int fdkod_set_decimation_net(fdkod_plan_t *plan, const float *w, int n) {
    if (!plan) return FDKOD_ERR_INVALID_ARG;
    PlanImpl &p = plan->impl;
    if (!w) {
        cudaFree(p.net);
        p.net = nullptr;
        return FDKOD_OK;
    }
    if (n != fdkod::kNetSize) return FDKOD_ERR_INVALID_ARG;
    for (int i = 0; i < n; ++i)
        if (!std::isfinite(w[i]) || std::fabs(w[i]) > 3.0e38f) return FDKOD_ERR_INVALID_ARG;
    if (p.D < 2 || p.D > fdkod::kNetMaxD) return FDKOD_ERR_UNSUPPORTED;
    if (!p.net) {
        cudaError_t e = cudaMalloc(&p.net, sizeof(fdkod::NetWeights));
        if (e != cudaSuccess) {
            p.net = nullptr;
            return fdkod::net_status(e);
        }
    }
    for (int i = 0; i < n; ++i) p.net_host[i] = fdkod::bf16_value(fdkod::bf16_bits(w[i]));
    return fdkod::net_status(fdkod::upload_net(p));
}

extern "C" int fdkod_get_decimation_net(const fdkod_plan_t *plan, float *w, int cap) {
    if (!plan || (cap > 0 && !w)) return FDKOD_ERR_INVALID_ARG;
    const PlanImpl &p = plan->impl;
    if (!p.net) return 0;
    for (int i = 0; i < fdkod::kNetSize && i < cap; ++i) w[i] = p.net_host[i];
    return fdkod::kNetSize;
}

extern "C" int fdkod_net_adjoint(fdkod_plan_t *plan, const float *vol_slice, const float *ref_slice, int z,
                                 float *dS, float *sq_err, uintptr_t stream) {
    if (!plan || !vol_slice || !ref_slice || !dS || !sq_err) return FDKOD_ERR_INVALID_ARG;
    PlanImpl &p = plan->impl;
    if (p.D < 2 || z < 0 || z >= p.g.N) return FDKOD_ERR_INVALID_ARG;
    const int N = p.g.N;
    dim3 grid((unsigned)((N + 15) / 16), (unsigned)((N + 15) / 16));
    fdkod::net_adjoint_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>(
        vol_slice, ref_slice, z, dS, sq_err, p.od.geo, p.od.w0, p.od.T, N, p.s, p.g.P, p.D, p.Pd, p.g.Nv, p.Tstride,
        (float)(M_PI / (double)p.Pd));
    return fdkod::net_status(cudaGetLastError());
}

extern "C" int fdkod_net_backward(fdkod_plan_t *plan, const void *Q, const float *w, const float *dS, int row_lo,
                                  int row_hi, float *dW, uintptr_t stream) {
    if (!plan || !Q || !w || !dS || !dW) return FDKOD_ERR_INVALID_ARG;
    PlanImpl &p = plan->impl;
    if (p.D < 2 || p.D > fdkod::kNetMaxD) return FDKOD_ERR_UNSUPPORTED;
    if (row_lo < 0 || row_hi > p.g.Nv || row_lo > row_hi) return FDKOD_ERR_INVALID_ARG;
    if (row_lo == row_hi) return FDKOD_OK;
    cudaStream_t st = (cudaStream_t)stream;
    switch (p.qtype) {
        case FDKOD_F32:
            return fdkod::net_status(fdkod::launch_backward_t(p, (const float *)Q, w, dS, row_lo, row_hi, dW, st));
        case FDKOD_BF16:
            return fdkod::net_status(
                fdkod::launch_backward_t(p, (const __nv_bfloat16 *)Q, w, dS, row_lo, row_hi, dW, st));
        case FDKOD_F16:
            return fdkod::net_status(fdkod::launch_backward_t(p, (const __half *)Q, w, dS, row_lo, row_hi, dW, st));
    }
    return FDKOD_ERR_INVALID_ARG;
}
