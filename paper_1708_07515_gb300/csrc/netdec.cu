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
// output views.  Per chunk it interpolates the shifted samples x from Q
// (FP32), runs layer 1 on the CUDA cores (FP32, BF16 weights) and stores a1
// as BF16 in the K-major operand layout of tc5.cuh, one MMA row per (view,
// column).  Layer 2 is 8 tiles of 128 rows x 16 channels on the tensor cores:
// per tile, five tcgen05.mma of K = 16 input channels, one per tap, whose A
// operand is the a1 block started 16 m rows (m views) further down -- the
// taps cost no data movement -- accumulating FP32 in tensor memory.  The
// plain low-pass runs on the CUDA cores while the MMAs do; then each thread
// reads its row of the accumulator (tcgen05.ld), applies the ReLU and adds
// its layer-3 terms to the output views it feeds.
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
constexpr int kKA = kTiles * kTileViews;   // a2 views per chunk
constexpr int kNA1 = kKA + 4;          // a1 views per chunk (two each side)
constexpr int kPlaneA1 = kNA1 * kG * 16;   // bytes of one K plane of a1
constexpr int kNetThreads = 128;
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

struct NetChunk {
    int J;    // output views per chunk
    int XL;   // x views before the chunk's first output view
    int NX;   // x views per chunk
};

__host__ __device__ inline NetChunk net_chunk(int D, int HD) {
    NetChunk c;
    c.J = (kKA - 5) / D + 1;
    c.XL = HD - 1 > 6 ? HD - 1 : 6;
    const int a = kNA1 + c.XL - 2, b = (c.J - 1) * D + HD + c.XL;
    c.NX = a > b ? a : b;
    return c;
}

// dynamic shared memory of net_decompose_kernel (bytes, after 128-byte alignment)
__host__ __device__ inline size_t net_smem(const NetChunk &c, int HD) {
    return 2 * (size_t)kPlaneA1 + sizeof(uint16_t) * kK * 256 + sizeof(float) * (size_t)c.NX * kG +
           sizeof(float) * (size_t)c.J * kG + sizeof(float) * 2 * kC * kK + sizeof(float) * (size_t)HD;
}

template <typename TQ>
__global__ void __launch_bounds__(kNetThreads, 4)
net_decompose_kernel(const TQ *__restrict__ Q, float *__restrict__ out, const int32_t *__restrict__ crop,
                     const GeomEntry *__restrict__ geo, const int32_t *__restrict__ Tq,
                     const NetWeights *__restrict__ net, int *status, int Tstride, int P, int D, int Pd, int HD,
                     int nrows, int Nu, int ngroups) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char *base = smem_raw + ((128u - (tma::smem_u32(smem_raw) & 127u)) & 127u);
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t tmem_slot;

    const int q = blockIdx.x / ngroups, grp = blockIdx.x - q * ngroups;
    const int v = blockIdx.y;
    const int t0 = grp * kG;
    const int T = __ldg(Tq + q);
    const size_t jstride = (size_t)nrows * Tstride;
    float *outq = out + ((size_t)q * Pd * nrows + v) * Tstride;
    const int tid = threadIdx.x;
    if (t0 >= T) {  // past this square's row length: zeros (uniform per CTA)
        for (int i = tid; i < Pd * kG; i += kNetThreads) {
            const int j = i / kG, t = t0 + i % kG;
            if (t < Tstride) outq[(size_t)j * jstride + t] = 0.f;
        }
        return;
    }
    const NetChunk ch = net_chunk(D, HD);
    unsigned char *a1 = base;                                       // 2 planes
    unsigned char *w2 = a1 + 2 * kPlaneA1;                          // kK blocks of 512 bytes
    float *xs = (float *)(w2 + sizeof(uint16_t) * kK * 256);        // [NX][kG]
    float *yacc = xs + (size_t)ch.NX * kG;                          // [J][kG]
    float *w1s = yacc + (size_t)ch.J * kG;                          // [kC][kK]
    float *w3s = w1s + kC * kK;                                     // [kC][kK]
    float *hs = w3s + kC * kK;                                      // [HD]

    for (int i = tid; i < kK * 256 / 8; i += kNetThreads)
        ((uint4 *)w2)[i] = ((const uint4 *)net->w2)[i];
    for (int i = tid; i < kC * kK; i += kNetThreads) {
        w1s[i] = net->w1[i];
        w3s[i] = net->w3[i];
    }
    for (int i = tid; i < HD; i += kNetThreads) hs[i] = net->h[i];
    if (tid == 0) {
        tma::mbar_init(&bar, 1);
        tma::fence_mbar_init();
    }
    if (tid < 32) tc5::alloc(&tmem_slot, kTmemCols);
    tc5::fence_before_sync();
    __syncthreads();
    tc5::fence_after_sync();
    const uint32_t tmem = tmem_slot;
    const int warp = tid >> 5, lane = tid & 31;
    const uint32_t sa1 = tma::smem_u32(a1), sw2 = tma::smem_u32(w2);
    constexpr uint32_t kIdesc = tc5::idesc_bf16_f32(128, 16);
    const int nchunks = (Pd + ch.J - 1) / ch.J;
    bool failed = false;
    uint32_t fail_parity = 0;

    for (int cc = 0; cc < nchunks; ++cc) {
        const int j0 = cc * ch.J;
        const int Jc = min(ch.J, Pd - j0);
        const int kx0 = j0 * D - ch.XL;  // view of x[0]
        // 1. shifted samples
        for (int i = tid; i < ch.NX * kG; i += kNetThreads) {
            const int ix = i / kG, g = i - ix * kG;
            xs[i] = shifted_sample(Q, crop, geo, q, wrap(kx0 + ix, P), t0 + g, T, v, nrows, P, Nu);
        }
        __syncthreads();
        // 2. layer 1: a1 view ka (= view j0 D - 4 + ka), column g, as BF16
        {
            const int g = tid & (kG - 1);
            for (int ka = tid / kG; ka < kNA1; ka += kNetThreads / kG) {
                const float *xp = xs + (size_t)(ka + ch.XL - 6) * kG + g;
                const float x0 = xp[0], x1 = xp[kG], x2 = xp[2 * kG], x3 = xp[3 * kG], x4 = xp[4 * kG];
                uint32_t pk[8];
#pragma unroll
                for (int c = 0; c < kC; c += 2) {
                    const float *wa = w1s + c * kK, *wb = wa + kK;
                    float za = wa[0] * x0, zb = wb[0] * x0;
                    za = fmaf(wa[1], x1, za);
                    zb = fmaf(wb[1], x1, zb);
                    za = fmaf(wa[2], x2, za);
                    zb = fmaf(wb[2], x2, zb);
                    za = fmaf(wa[3], x3, za);
                    zb = fmaf(wb[3], x3, zb);
                    za = fmaf(wa[4], x4, za);
                    zb = fmaf(wb[4], x4, zb);
                    const __nv_bfloat162 b2 = __floats2bfloat162_rn(fmaxf(za, 0.f), fmaxf(zb, 0.f));
                    pk[c / 2] = *(const uint32_t *)&b2;
                }
                const int r = ka * kG + g;
                *(uint4 *)(a1 + (size_t)r * 16) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
                *(uint4 *)(a1 + kPlaneA1 + (size_t)r * 16) = make_uint4(pk[4], pk[5], pk[6], pk[7]);
            }
        }
        tma::fence_proxy_async();
        tc5::fence_before_sync();
        __syncthreads();
        tc5::fence_after_sync();
        // 3. layer 2 on the tensor cores: tile i = a2 views 8i .. 8i + 7 of
        // the chunk (rows view * 16 + column); tap m reads a1 from row 16 m on
        if (tid == 0) {
#pragma unroll 1
            for (int i = 0; i < kTiles; ++i)
#pragma unroll
                for (int m = 0; m < kK; ++m)
                    tc5::mma_bf16(tmem + (uint32_t)(16 * i),
                                  tc5::smem_desc(sa1 + (uint32_t)((128 * i + 16 * m) * 16), kPlaneA1, 128),
                                  tc5::smem_desc(sw2 + (uint32_t)(512 * m), 256, 128), kIdesc, m > 0 ? 1u : 0u);
            tc5::commit(&bar);
        }
        // plain low-pass meanwhile: output view j0 + jl, column g
        for (int i = tid; i < Jc * kG; i += kNetThreads) {
            const int jl = i / kG, g = i - jl * kG;
            const float *xp = xs + (size_t)(jl * D + ch.XL) * kG + g;
            float acc = hs[0] * xp[0];
            for (int d = 1; d < HD; ++d) acc = fmaf(hs[d], xp[(size_t)d * kG] + xp[-(ptrdiff_t)d * kG], acc);
            yacc[i] = acc;
        }
        __syncthreads();
        const bool ok = tma::mbar_wait_bounded(&bar, (uint32_t)(cc & 1), kNetWaitNs);
        if (!__syncthreads_and(ok)) {
            failed = true;
            fail_parity = (uint32_t)(cc & 1);
            break;
        }
        tc5::fence_after_sync();
        // 4. layer 3: row (view 8 i + 2 warp + lane / 16, column lane % 16)
        {
            const int g = lane & (kG - 1);
#pragma unroll 1
            for (int i = 0; i < kTiles; ++i) {
                float z[16];
                tc5::ld16(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(16 * i), z);
                const int ka2 = kTileViews * i + 2 * warp + (lane >> 4);
                // output views jl with 0 <= ka2 - jl D <= 4
                int jl = ka2 >= 4 ? (ka2 - 4 + D - 1) / D : 0;
                for (; jl * D <= ka2 && jl < Jc; ++jl) {
                    const float *w = w3s + (ka2 - jl * D);
                    float p = 0.f;
#pragma unroll
                    for (int c = 0; c < kC; ++c) p = fmaf(w[c * kK], fmaxf(z[c], 0.f), p);
                    atomicAdd(yacc + jl * kG + g, p);
                }
            }
        }
        tc5::fence_before_sync();
        __syncthreads();
        // 5. store
        for (int i = tid; i < Jc * kG; i += kNetThreads) {
            const int jl = i / kG, t = t0 + (i - jl * kG);
            if (t < Tstride) outq[(size_t)(j0 + jl) * jstride + t] = yacc[i];
        }
    }
    if (failed) {
        // the MMAs never signalled: report, give them another bounded wait, leave
        if (tid == 0) atomicOr(status, 2);
        tma::mbar_wait_bounded(&bar, fail_parity, kNetWaitNs);
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
    const size_t smem = net_smem(ch, HD) + 128;
    cudaError_t e = ensure_smem<net_decompose_kernel<TQ>>(smem);
    if (e != cudaSuccess) return e;
    const int ngroups = (p.Tstride + kG - 1) / kG;
    dim3 grid((unsigned)(ngroups * p.od.nsq), (unsigned)nrows);
    net_decompose_kernel<TQ><<<grid, kNetThreads, smem, st>>>(Q, out, p.od.crop, p.od.geo, p.od.T, p.net, p.status,
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
    for (int i = 0; i < kC * kK; ++i) {
        h.w1[i] = W1[i];
        h.w3[i] = W3[i];
    }
    // tap m: B[n = c][k = c'] at byte (c' / 8) 256 + c 16 + (c' % 8) 2
    for (int m = 0; m < kK; ++m)
        for (int c = 0; c < kC; ++c)
            for (int ci = 0; ci < kC; ++ci)
                h.w2[m * 256 + (ci / 8) * 128 + c * 8 + (ci % 8)] = bf16_bits(W2[(c * kC + ci) * kK + m]);
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
