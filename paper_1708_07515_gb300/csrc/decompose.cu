// Decomposition stage of FDK-OD (Sec. 2.1): for every square q, detector row
// v and shifted column t, shift each view's row so the square centre sits
// on one column (linear interpolation at column phi_k + w0 + t, i.e. crop
// column c_qk + t with sub-pixel part f_qk), low-pass it along the view
// axis with symmetric taps h[|i|], |i| < H D (circular over the orbit; the
// triangle (D - |i|) / D^2 with H = 1 by default, a windowed sinc with
// H = 2 as an option) and keep every D-th view.  The views are streamed in
// order: view k = jD + r adds w[r][m] = h[|r + (H - 1 - m) D|] of its sample
// to decimated view j - H + 1 + m, m < 2H, so only 2H running sums are live
// (two for the triangle: (D - r) / D^2 to view j, r / D^2 to view j + 1).
// The stream starts H D - 1 views before view 0 and runs (H - 1) D views
// past the last one (both wrapped): every decimated view sees its whole
// support.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <type_traits>

#include "fdkod_internal.cuh"
#include "tma.cuh"

namespace fdkod {
namespace {

constexpr int kTX = 64, kTY = 4;

__device__ __forceinline__ float ld_q(const float *p) { return __ldg(p); }
__device__ __forceinline__ float ld_q(const __nv_bfloat16 *p) { return __bfloat162float(__ldg(p)); }
__device__ __forceinline__ float ld_q(const __half *p) { return __half2float(__ldg(p)); }

// floor(a / b) for b > 0
__host__ __device__ __forceinline__ int floor_div(int a, int b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }

// Generic path: one thread per (q, v, t), consecutive threads on consecutive
// t (each view's crop row is one coalesced segment).
template <typename TQ, int H>
__global__ void __launch_bounds__(kTX *kTY)
decompose_kernel(const TQ *__restrict__ Q, float *__restrict__ Sp, const int32_t *__restrict__ crop,
                 const GeomEntry *__restrict__ geo, const int32_t *__restrict__ Tq, const float4 *__restrict__ tapw,
                 int Tstride, int P, int D, int Pd, int Nv, int Nu) {
    const int t = blockIdx.x * kTX + threadIdx.x;
    const int v = blockIdx.y * kTY + threadIdx.y;
    const int q = blockIdx.z;
    if (t >= Tstride || v >= Nv) return;
    const size_t vstride = (size_t)Nv * Tstride;
    float *out = Sp + ((size_t)q * Pd * Nv + v) * Tstride + t;
    if (t >= Tq[q]) {
        for (int j = 0; j < Pd; ++j) out[(size_t)j * vstride] = 0.f;
        return;
    }
    const size_t qo = (size_t)q * P;
    const size_t row = (size_t)v * Nu;
    const size_t view = (size_t)Nv * Nu;
    auto sample = [&](int k) -> float {
        const int c = __ldg(crop + qo + k) + t;
        const float f = __ldg(&geo[qo + k].frac);
        const TQ *r = Q + (size_t)k * view + row;
        const float a = (c >= 0 && c < Nu) ? ld_q(r + c) : 0.f;
        const float b = (c + 1 >= 0 && c + 1 < Nu) ? ld_q(r + c + 1) : 0.f;
        return fmaf(f, b - a, a);
    };
    float acc[2 * H];
#pragma unroll
    for (int m = 0; m < 2 * H; ++m) acc[m] = 0.f;
    const int nstream = P + (2 * H - 1) * D - 1;
    const int kp0 = -(H * D - 1);
    int jb = floor_div(kp0, D), r = kp0 - jb * D, kk = ((kp0 % P) + P) % P;
    for (int pos = 0; pos < nstream; ++pos) {
        const float sm = sample(kk);
        const float4 w = __ldg(tapw + r);
        const float wm[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
        for (int m = 0; m < 2 * H; ++m) acc[m] = fmaf(wm[m], sm, acc[m]);
        if (r == D - 1) {
            const int jst = jb - H + 1;  // its support is complete
            if (jst >= 0) out[(size_t)jst * vstride] = acc[0];
#pragma unroll
            for (int m = 0; m < 2 * H - 1; ++m) acc[m] = acc[m + 1];
            acc[2 * H - 1] = 0.f;
            r = 0;
            ++jb;
        } else {
            ++r;
        }
        if (++kk == P) kk = 0;
    }
}


// ---------------------------------------------------------------------------
// TMA path: one CTA per (square q, band of VB detector rows), warp
// specialised.  The producer warp's lane 0 brings each view's crop box
// (VB rows x Wc columns starting at the 16-byte aligned column below
// crop[q][k]) into a ring of kStages slots of kG views (Ring<TQ>) with 3D
// bulk-tensor copies (zero fill outside the detector); slot n is full when
// its bytes have landed (mbarrier full[n]) and free again when all consumer
// warps have arrived on empty[n].  No block-wide barrier inside the view loop.
//
// Consumers: LPR lanes share a pair of adjacent detector rows and each lane
// owns C consecutive columns t0 .. t0 + C - 1 of both (rows_per_lane), so one
// view costs the lane a few vector shared loads at compile-time offsets per
// row (the column offset of the crop inside its aligned box selects one of
// four code paths, uniform per view) and, per column, one lerp and the 2H
// tap FMAs; the per-view bookkeeping is shared by the two rows.  Everything else
// a view needs -- shift fraction, which tap weights apply and whether a
// decimated view is complete -- is one 8-byte entry of a per-CTA table in
// stream order, built once from crop[q][.] and frac[q][.], plus the weights
// w[r] of its block offset r (one 16-byte entry per r).

constexpr int kConsumerWarps = 8;
// adjacent detector rows per lane (the per-view work is shared): two with
// the triangle's two running sums, one with the four of 2D-tap filters
// (registers; measured)
__host__ __device__ constexpr int rows_per_lane(int H) { return H == 1 ? 2 : 1; }
// ring shape per element type (measured): slots of kG views, kStages slots
template <typename TQ>
struct Ring {
    static constexpr int kG = sizeof(TQ) == 4 ? 2 : 4;
    static constexpr int kStages = 3;
};
constexpr int kDecThreads = 32 * (kConsumerWarps + 1);
constexpr int kRingSlack = 128;  // bytes after the ring: vector loads of the last row may run past its end
constexpr uint64_t kDecWaitNs = 2000000000ull;

// code word of a table entry: bits 0-2 the crop's offset inside its aligned
// box, bit 3 "last view of a decimated block" (rotate the running sums),
// bits 4-11 the block offset r (its weights), bits 12.. the decimated view
// to store plus one (0: none, a view before view 0).  D <= 128.
constexpr int kCodeRotate = 8, kCodeTapShift = 4, kCodeStoreShift = 12;

// Per-CTA tables over the stream positions pos = 0 .. P + (2H - 1) D - 2
// (view k' = pos - (H D - 1), taken mod P): s_fc[pos] = {shift fraction of
// square q, code word}, s_c[pos] = crop column, and s_taps[r] = the 2H
// running-sum weights of block offset r (tapw, r < D).
template <int kAl>
__device__ __forceinline__ void build_stream_table(float2 *s_fc, int *s_c, float4 *s_taps,
                                                   const int32_t *__restrict__ crop,
                                                   const GeomEntry *__restrict__ geo,
                                                   const float4 *__restrict__ tapw, int q, int P, int D, int Pd,
                                                   int H) {
    const int nstream = P + (2 * H - 1) * D - 1;
    for (int pos = threadIdx.x; pos < nstream; pos += blockDim.x) {
        const int kp = pos - (H * D - 1);
        const int kk = ((kp % P) + P) % P;
        const int c = crop[(size_t)q * P + kk];
        const int jb = floor_div(kp, D);
        const int r = kp - jb * D;
        int code = (c & (kAl - 1)) | (r << kCodeTapShift);
        const int jst = jb - H + 1;  // decimated view whose support ends here
        if (r == D - 1) code |= kCodeRotate | (jst >= 0 && jst < Pd ? (jst + 1) << kCodeStoreShift : 0);
        s_fc[pos] = make_float2(geo[(size_t)q * P + kk].frac, __int_as_float(code));
        s_c[pos] = c;
    }
    for (int r = threadIdx.x; r < D; r += blockDim.x) s_taps[r] = tapw[r];
}

// NV vectors of 4 consecutive elements from 32-bit shared address a, widened to float
template <typename TQ, int NV>
struct VecLoad;
template <int NV>
struct VecLoad<float, NV> {
    static __device__ __forceinline__ void f(uint32_t a, float *e) {
#pragma unroll
        for (int k = 0; k < NV; ++k)
            asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                         : "=f"(e[4 * k]), "=f"(e[4 * k + 1]), "=f"(e[4 * k + 2]), "=f"(e[4 * k + 3])
                         : "r"(a + 16u * k)
                         : "memory");
    }
};
template <int NV>
struct VecLoad<__nv_bfloat16, NV> {
    static __device__ __forceinline__ void f(uint32_t a, float *e) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            uint32_t w0, w1;
            asm volatile("ld.shared.v2.b32 {%0, %1}, [%2];" : "=r"(w0), "=r"(w1) : "r"(a + 8u * k) : "memory");
            // bfloat16 is the top half of a float32
            e[4 * k] = __uint_as_float(w0 << 16);
            e[4 * k + 1] = __uint_as_float(w0 & 0xffff0000u);
            e[4 * k + 2] = __uint_as_float(w1 << 16);
            e[4 * k + 3] = __uint_as_float(w1 & 0xffff0000u);
        }
    }
};
template <int NV>
struct VecLoad<__half, NV> {
    static __device__ __forceinline__ void f(uint32_t a, float *e) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            uint32_t w0, w1;
            asm volatile("ld.shared.v2.b32 {%0, %1}, [%2];" : "=r"(w0), "=r"(w1) : "r"(a + 8u * k) : "memory");
            const float2 p0 = __half22float2(*reinterpret_cast<const __half2 *>(&w0));
            const float2 p1 = __half22float2(*reinterpret_cast<const __half2 *>(&w1));
            e[4 * k] = p0.x;
            e[4 * k + 1] = p0.y;
            e[4 * k + 2] = p1.x;
            e[4 * k + 3] = p1.y;
        }
    }
};

// One view for one lane: in each of its RPL rows (row stride rs bytes),
// columns t0 + i (i < C) sample the row at box column O + i (+ the shift
// fraction f) and feed that row's 2H running sums with weights w.
template <typename TQ, int C, int O, int H, int RPL>
__device__ __forceinline__ void view_cols(uint32_t a, uint32_t rs, float f, float4 w, float (*acc)[2 * H][C]) {
    constexpr int NV = (O + C) / 4 + 1;  // vectors covering elements O .. O + C
#pragma unroll
    for (int r = 0; r < RPL; ++r) {
        float e[4 * NV];
        VecLoad<TQ, NV>::f(a + rs * (uint32_t)r, e);
#pragma unroll
        for (int i = 0; i < C; ++i) {
            const float a0 = e[O + i], a1 = e[O + i + 1];
            const float smp = fmaf(f, a1 - a0, a0);
            acc[r][0][i] = fmaf(w.x, smp, acc[r][0][i]);
            acc[r][1][i] = fmaf(w.y, smp, acc[r][1][i]);
            if (H == 2) {
                acc[r][2][i] = fmaf(w.z, smp, acc[r][2][i]);
                acc[r][3][i] = fmaf(w.w, smp, acc[r][3][i]);
            }
        }
    }
}

// off: the crop's offset inside its 16-byte aligned box (elements).  For
// 16-bit data the vectors are 8 bytes, so the lane's address moves by whole
// vectors and the remainder (0..3) picks the code path.
template <typename TQ, int C, int H, int RPL>
__device__ __forceinline__ void view_step(uint32_t a, uint32_t rs, int off, float f, float4 w,
                                          float (*acc)[2 * H][C]) {
    if (sizeof(TQ) == 2) a += 8u * (uint32_t)(off >> 2);
    switch (off & 3) {
        case 0: view_cols<TQ, C, 0, H, RPL>(a, rs, f, w, acc); break;
        case 1: view_cols<TQ, C, 1, H, RPL>(a, rs, f, w, acc); break;
        case 2: view_cols<TQ, C, 2, H, RPL>(a, rs, f, w, acc); break;
        default: view_cols<TQ, C, 3, H, RPL>(a, rs, f, w, acc); break;
    }
}

template <typename TQ, int C, int LPR, int H>
__global__ void __launch_bounds__(kDecThreads)
decompose_tma_kernel(const __grid_constant__ CUtensorMap tmap, float *__restrict__ Sp,
                     const int32_t *__restrict__ crop, const GeomEntry *__restrict__ geo,
                     const int32_t *__restrict__ Tq, const float4 *__restrict__ tapw, int *status, int Tstride, int P,
                     int D, int Pd, int Nv, int Wc, int tile_stride) {
    constexpr int ES = (int)sizeof(TQ);
    constexpr int kAlign = 16 / ES;
    constexpr int kG = Ring<TQ>::kG, kStages = Ring<TQ>::kStages;
    constexpr int RPL = rows_per_lane(H);
    constexpr int RPW = 32 / LPR * RPL;        // detector rows per consumer warp
    constexpr int VB = kConsumerWarps * RPW;   // rows per CTA (box height)
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char *ring = smem_raw + ((128u - (tma::smem_u32(smem_raw) & 127u)) & 127u);
    const uint32_t tile_bytes = (uint32_t)(ES * tile_stride);
    // views streamed: k' = -(H D - 1) .. P - 1 + (H - 1) D (view k' mod P)
    const int nstream = P + (2 * H - 1) * D - 1;
    const int nstage = (nstream + kG - 1) / kG;
    float4 *s_taps = (float4 *)(ring + (size_t)tile_bytes * kStages * kG + kRingSlack);
    float2 *s_fc = (float2 *)(s_taps + D);
    int *s_c = (int *)(s_fc + nstream);
    __shared__ __align__(8) uint64_t full[kStages], empty[kStages];

    const int q = blockIdx.x;
    const int v0 = blockIdx.y * VB;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;

    build_stream_table<kAlign>(s_fc, s_c, s_taps, crop, geo, tapw, q, P, D, Pd, H);
    if (threadIdx.x == 0) {
        for (int i = 0; i < kStages; ++i) {
            tma::mbar_init(&full[i], 1);
            tma::mbar_init(&empty[i], kConsumerWarps);
        }
        tma::fence_mbar_init();
    }
    __syncthreads();

    if (ty == kConsumerWarps) {  // producer
        if (tx != 0) return;
        int kk = ((-(H * D - 1)) % P + P) % P, n = 0, slot = 0;
        uint32_t phase = 0;  // parity of the slot's current round
        for (; n < nstage; ++n) {
            // round r of a slot may start once its round r - 1 was consumed
            if (n >= kStages && !tma::mbar_wait_bounded(&empty[slot], phase ^ 1u, kDecWaitNs)) {
                atomicOr(status, 2);
                break;
            }
            const int nv = min(kG, nstream - n * kG);
            tma::fence_proxy_async();
            tma::mbar_arrive_expect_tx(&full[slot], (uint32_t)(nv * VB * Wc * ES));
            for (int w = 0; w < nv; ++w) {
                tma::load_3d(ring + (size_t)tile_bytes * (slot * kG + w), &tmap, &full[slot],
                             s_c[n * kG + w] & ~(kAlign - 1), v0, kk);
                if (++kk == P) kk = 0;
            }
            if (++slot == kStages) {
                slot = 0;
                phase ^= 1u;
            }
        }
        // copies still in flight must land before the CTA may exit
        for (int m = max(0, n - kStages); m < n; ++m)
            tma::mbar_wait_bounded(&full[m % kStages], (uint32_t)((m / kStages) & 1), kDecWaitNs);
        return;
    }

    const int rib = (ty * (32 / LPR) + tx / LPR) * RPL;  // first of the lane's rows in the band
    const int t0 = (tx % LPR) * C;                      // first column of the lane
    const int v = v0 + rib;
    const int T = Tq[q];
    const bool act = t0 < T;
    const bool store = t0 < Tstride;
    float acc[RPL][2 * H][C];
#pragma unroll
    for (int r = 0; r < RPL; ++r)
#pragma unroll
        for (int m = 0; m < 2 * H; ++m)
#pragma unroll
            for (int i = 0; i < C; ++i) acc[r][m][i] = 0.f;
    const size_t vstride = (size_t)Nv * Tstride;
    float *out = Sp + ((size_t)q * Pd * Nv + v) * Tstride + t0;  // row v; row v + r is r Tstride further
    const uint32_t lane_addr = tma::smem_u32(ring) + (uint32_t)(ES * (rib * Wc + t0));
    const uint32_t row_bytes = (uint32_t)(ES * Wc);
    int slot = 0;
    uint32_t phase = 0;

    for (int n = 0; n < nstage; ++n) {
        const bool ok = tma::mbar_wait_bounded(&full[slot], phase, kDecWaitNs);
        if (!__all_sync(0xffffffffu, ok)) {
            if (tx == 0) atomicOr(status, 2);
            return;
        }
        const int nv = min(kG, nstream - n * kG);
        const uint32_t sa = lane_addr + tile_bytes * (uint32_t)(slot * kG);
#pragma unroll
        for (int w = 0; w < kG; ++w) {
            if (w < nv) {
                const float2 fc = s_fc[n * kG + w];
                const int code = __float_as_int(fc.y);
                const float4 tp = s_taps[(code >> kCodeTapShift) & 255];
                if (act)
                    view_step<TQ, C, H, RPL>(sa + tile_bytes * (uint32_t)w, row_bytes, code & (kAlign - 1), fc.x, tp,
                                             acc);
                if (code & kCodeRotate) {
                    const int jst = (code >> kCodeStoreShift) - 1;
                    if (jst >= 0 && store) {
#pragma unroll
                        for (int r = 0; r < RPL; ++r) {
                            if (v + r < Nv) {
                                float o[C];
#pragma unroll
                                for (int i = 0; i < C; ++i) o[i] = t0 + i < T ? acc[r][0][i] : 0.f;
                                float4 *dst = (float4 *)(out + (size_t)jst * vstride + (size_t)r * Tstride);
#pragma unroll
                                for (int i = 0; i < C / 4; ++i)  // Tstride is a multiple of 4
                                    if (t0 + 4 * i < Tstride)
                                        dst[i] = make_float4(o[4 * i], o[4 * i + 1], o[4 * i + 2], o[4 * i + 3]);
                            }
                        }
                    }
#pragma unroll
                    for (int r = 0; r < RPL; ++r)
#pragma unroll
                        for (int i = 0; i < C; ++i) {
#pragma unroll
                            for (int m = 0; m < 2 * H - 1; ++m) acc[r][m][i] = acc[r][m + 1][i];
                            acc[r][2 * H - 1][i] = 0.f;
                        }
                }
            }
        }
        __syncwarp();
        if (tx == 0) tma::mbar_arrive(&empty[slot]);
        if (++slot == kStages) {
            slot = 0;
            phase ^= 1u;
        }
    }
}

// columns per lane C and lanes per row LPR from the decomposed row length
struct DecShape {
    int C, LPR;
};
inline DecShape dec_shape(int Tstride) {
    if (Tstride <= 32) return {4, 8};
    if (Tstride <= 64) return {4, 16};
    if (Tstride <= 128) return {4, 32};
    return {8, 32};
}

template <typename TQ, int C, int LPR, int H>
cudaError_t launch_tma_shape(const PlanImpl &p, const CUtensorMap &map, float *out, int Wc, cudaStream_t st,
                             int nrows, size_t smem, int tile_stride) {
    cudaError_t e = ensure_smem<decompose_tma_kernel<TQ, C, LPR, H>>(smem);
    if (e != cudaSuccess) return e;
    constexpr int VB = kConsumerWarps * (32 / LPR) * rows_per_lane(H);
    dim3 grid(p.od.nsq, (nrows + VB - 1) / VB);
    decompose_tma_kernel<TQ, C, LPR, H><<<grid, kDecThreads, smem, st>>>(map, out, p.od.crop, p.od.geo, p.od.T,
                                                                         p.tapw, p.status, p.Tstride, p.g.P, p.D,
                                                                         p.Pd, nrows, Wc, tile_stride);
    return cudaGetLastError();
}

template <typename TQ, int H>
cudaError_t launch_tma_h(const PlanImpl &p, const CUtensorMap &map, float *out, int Wc, cudaStream_t st, int nrows,
                         size_t smem, int tile_stride, DecShape sh) {
    if (sh.C == 8) return launch_tma_shape<TQ, 8, 32, H>(p, map, out, Wc, st, nrows, smem, tile_stride);
    if (sh.LPR == 32) return launch_tma_shape<TQ, 4, 32, H>(p, map, out, Wc, st, nrows, smem, tile_stride);
    if (sh.LPR == 16) return launch_tma_shape<TQ, 4, 16, H>(p, map, out, Wc, st, nrows, smem, tile_stride);
    return launch_tma_shape<TQ, 4, 8, H>(p, map, out, Wc, st, nrows, smem, tile_stride);
}

// TMA applies when Q's rows are whole 16-byte units, Q and S' are 16-byte
// aligned (vector stores), a crop box (T_max + one interpolation neighbour +
// alignment) fits 256 columns, D <= 128 and the ring plus the stream tables
// fit in shared memory.
template <typename TQ>
cudaError_t try_tma(const PlanImpl &p, const TQ *Q, float *out, cudaStream_t st, int nrows, bool &launched) {
    launched = false;
    constexpr int kAlign = 16 / (int)sizeof(TQ);
    if ((p.g.Nu % kAlign) != 0 || ((uintptr_t)Q & 15) != 0 || ((uintptr_t)out & 15) != 0) return cudaSuccess;
    const int Wc = (p.od.Tmax + 1 + (kAlign - 1) + (kAlign - 1)) & ~(kAlign - 1);
    if (Wc > 256 || p.Tstride > 256 || p.D > kMaxTapD) return cudaSuccess;  // block offset: 8 bits of the code
    const DecShape sh = dec_shape(p.Tstride);
    const int VB = kConsumerWarps * (32 / sh.LPR) * rows_per_lane(p.tap_blocks);
    const int tile_stride = (VB * Wc + 63) & ~63;  // elements; 128-byte multiple for every type
    const int nstream = p.g.P + (2 * p.tap_blocks - 1) * p.D - 1;
    const size_t smem = 128 + sizeof(TQ) * (size_t)Ring<TQ>::kStages * Ring<TQ>::kG * tile_stride + kRingSlack +
                        16 * (size_t)p.D +
                        12 * (size_t)nstream;
    if (smem > 200 * 1024) return cudaSuccess;
    CUtensorMap map;
    const uint64_t dims[3] = {(uint64_t)p.g.Nu, (uint64_t)nrows, (uint64_t)p.g.P};
    const uint64_t strides[2] = {(uint64_t)p.g.Nu * sizeof(TQ), (uint64_t)p.g.Nu * nrows * sizeof(TQ)};
    const uint32_t box[3] = {(uint32_t)Wc, (uint32_t)VB, 1u};
    const CUtensorMapDataType dt = sizeof(TQ) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                   : (std::is_same<TQ, __half>::value ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                                                      : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16);
    if (encode_map_3d(&map, dt, Q, dims, strides, box) != cudaSuccess) return cudaSuccess;
    launched = true;
    if (p.tap_blocks == 2) return launch_tma_h<TQ, 2>(p, map, out, Wc, st, nrows, smem, tile_stride, sh);
    return launch_tma_h<TQ, 1>(p, map, out, Wc, st, nrows, smem, tile_stride, sh);
}

template <typename TQ>
cudaError_t launch_t(const PlanImpl &p, const TQ *Q, float *out, cudaStream_t st, int nrows) {
    if (p.tap_blocks != 1 && p.tap_blocks != 2) return cudaErrorInvalidValue;
    bool launched = false;
    cudaError_t te = try_tma(p, Q, out, st, nrows, launched);
    if (launched || te != cudaSuccess) return te;
    dim3 grid((p.Tstride + kTX - 1) / kTX, (nrows + kTY - 1) / kTY, p.od.nsq);
    if (p.tap_blocks == 2)
        decompose_kernel<TQ, 2><<<grid, dim3(kTX, kTY), 0, st>>>(Q, out, p.od.crop, p.od.geo, p.od.T, p.tapw,
                                                                 p.Tstride, p.g.P, p.D, p.Pd, nrows, p.g.Nu);
    else
        decompose_kernel<TQ, 1><<<grid, dim3(kTX, kTY), 0, st>>>(Q, out, p.od.crop, p.od.geo, p.od.T, p.tapw,
                                                                 p.Tstride, p.g.P, p.D, p.Pd, nrows, p.g.Nu);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_decompose(const PlanImpl &p, const void *Q, float *out, cudaStream_t st, Band b) {
    const int nrows = b.nrows < 0 ? p.g.Nv : b.nrows;
    if (p.net) return launch_net_decompose(p, Q, out, st, nrows);
    switch (p.qtype) {
        case FDKOD_F32: return launch_t(p, (const float *)Q, out, st, nrows);
        case FDKOD_BF16: return launch_t(p, (const __nv_bfloat16 *)Q, out, st, nrows);
        case FDKOD_F16: return launch_t(p, (const __half *)Q, out, st, nrows);
    }
    return cudaErrorInvalidValue;
}

}  // namespace fdkod
