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
#include <utility>

#include "fdkod_internal.cuh"
#include "packed.cuh"
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
                 int Tstride, int P, int D, int Pd, int Nv, int Nu, int rowoff, int rowend) {
    const int t = blockIdx.x * kTX + threadIdx.x;
    const int v = rowoff + blockIdx.y * kTY + threadIdx.y;
    const int q = blockIdx.z;
    if (t >= Tstride || v >= rowend) return;
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
// Consumers: the 32 lanes of a warp share its rows (rows_per_lane adjacent
// detector rows) and lane l owns the columns l, l + 32, ... (C of them), so
// per view and column a lane makes two scalar shared loads at the crop's
// offset inside its aligned box plus compile-time offsets -- consecutive
// lanes read consecutive elements, free of bank conflicts for every offset
// -- one lerp and the 2H tap FMAs; the per-view bookkeeping is shared by the
// lane's rows and columns.  (Lanes that owned C consecutive columns loaded
// them as aligned vectors and picked the offset's code path per view: about
// 20 instructions per shifted sample, issue-bound.)  Everything else
// a view needs -- shift fraction, which tap weights apply and whether a
// decimated view is complete -- is one 8-byte entry of a per-CTA table in
// stream order, built once from crop[q][.] and frac[q][.], plus the weights
// w[r] of its block offset r (one 16-byte entry per r).

constexpr int kConsumerWarps = 8;
// adjacent detector rows per lane (the per-view bookkeeping -- table loads,
// slot waits, decimated-view stores -- is shared by them): four with the
// triangle's two running sums, two with the four of 2D-tap filters
// (registers; measured: 2 -> 4 rows took 1.63 -> 1.48 ms at 512^3); half of
// that where the launch would not fill two waves of the GPU (short row bands)
__host__ __device__ constexpr int rows_per_lane(int H, bool wide = true) {
    return (H == 1 ? 4 : 2) / (wide ? 1 : 2);
}
// ring shape per element type (measured): slots of kG views, kStages slots
template <typename TQ>
struct Ring {
    static constexpr int kG = sizeof(TQ) == 4 ? 2 : 4;
    static constexpr int kStages = 3;
};
constexpr int kDecThreads = 32 * (kConsumerWarps + 1);
// bytes after the ring: a lane's columns run up to 32 C + 1 elements (plus
// the crop's offset, < 16 bytes) past its row's start, beyond the last row's
// Wc columns; rounded up to 128 bytes so the tables behind it (float4 and
// float2 entries) stay aligned
__host__ __device__ constexpr int kColSlack(int C) { return (4 * (32 * C + 1) + 16 + 127) & ~127; }
static_assert(kColSlack(1) % 16 == 0 && kColSlack(8) % 16 == 0, "table alignment");
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

// One element at a compile-time byte offset from 32-bit shared address a,
// widened to float.
template <typename TQ, int OFF>
struct Ld1;
template <int OFF>
struct Ld1<float, OFF> {
    static __device__ __forceinline__ float f(uint32_t a) {
        float v;
        asm volatile("ld.shared.f32 %0, [%1+%2];" : "=f"(v) : "r"(a), "n"(OFF) : "memory");
        return v;
    }
};
template <int OFF>
struct Ld1<__nv_bfloat16, OFF> {
    static __device__ __forceinline__ float f(uint32_t a) {
        uint32_t u;
        asm volatile("ld.shared.u16 %0, [%1+%2];" : "=r"(u) : "r"(a), "n"(OFF) : "memory");
        return __uint_as_float(u << 16);  // bfloat16 is the top half of a float32
    }
};
template <int OFF>
struct Ld1<__half, OFF> {
    static __device__ __forceinline__ float f(uint32_t a) {
        unsigned short h;
        asm volatile("ld.shared.u16 %0, [%1+%2];" : "=h"(h) : "r"(a), "n"(OFF) : "memory");
        return __half2float(__ushort_as_half(h));
    }
};

// One view for one lane: in each of its RPL rows (row stride rs bytes), the
// columns t = lane + 32 i (i < C, t < T) sample the row at box column
// off + t (+ the shift fraction f) and feed that row's 2H running sums with
// weights w.  a is the byte address of box column off + lane of the lane's
// first row, so consecutive lanes read consecutive elements (no bank
// conflicts) whatever the crop's offset off inside its aligned box.
// Columns past T are computed too (no branch; their sums are never stored):
// their loads stay inside the CTA's shared memory, within the next row, the
// next slot or the ring's tail slack of kColSlack(C) bytes.
//
// Rows are taken in pairs (r, r + 1) where the lane has an even number of
// them: the two rows share the shift fraction and the tap weights, so one
// packed two-lane FP32 instruction (each lane rounded as the scalar
// operation would be) does the work of two.  acc[rp][m][i] holds running
// sum m of column i for rows 2 rp (x) and 2 rp + 1 (y); a lane with one row
// uses x only.
template <typename TQ, int I, int C, int H>
__device__ __forceinline__ void col_step(uint32_t ar, float f, float4 w, float2 (&acc)[2 * H][C]) {
    constexpr int ES = (int)sizeof(TQ);
    const float a0 = Ld1<TQ, ES * 32 * I>::f(ar), a1 = Ld1<TQ, ES * (32 * I + 1)>::f(ar);
    const float smp = fmaf(f, a1 - a0, a0);
    acc[0][I].x = fmaf(w.x, smp, acc[0][I].x);
    acc[1][I].x = fmaf(w.y, smp, acc[1][I].x);
    if (H == 2) {
        acc[2][I].x = fmaf(w.z, smp, acc[2][I].x);
        acc[3][I].x = fmaf(w.w, smp, acc[3][I].x);
    }
}

template <typename TQ, int I, int C, int H>
__device__ __forceinline__ void col_step2(uint32_t ar, uint32_t ar2, float2 f2, const float2 (&w2)[2 * H],
                                          float2 (&acc)[2 * H][C]) {
    constexpr int ES = (int)sizeof(TQ);
    const float2 a0 = make_float2(Ld1<TQ, ES * 32 * I>::f(ar), Ld1<TQ, ES * 32 * I>::f(ar2));
    const float2 a1 = make_float2(Ld1<TQ, ES * (32 * I + 1)>::f(ar), Ld1<TQ, ES * (32 * I + 1)>::f(ar2));
    // a0 + f (a1 - a0)
    const float2 smp = __ffma2_rn(f2, fsub2(a1, a0), a0);
#pragma unroll
    for (int m = 0; m < 2 * H; ++m) acc[m][I] = __ffma2_rn(w2[m], smp, acc[m][I]);
}

template <typename TQ, int C, int H, int... I>
__device__ __forceinline__ void row_cols(uint32_t ar, float f, float4 w, float2 (&acc)[2 * H][C],
                                         std::integer_sequence<int, I...>) {
    (col_step<TQ, I, C, H>(ar, f, w, acc), ...);
}

template <typename TQ, int C, int H, int... I>
__device__ __forceinline__ void row_pair_cols(uint32_t ar, uint32_t ar2, float2 f2, const float2 (&w2)[2 * H],
                                              float2 (&acc)[2 * H][C], std::integer_sequence<int, I...>) {
    (col_step2<TQ, I, C, H>(ar, ar2, f2, w2, acc), ...);
}

template <typename TQ, int C, int H, int RPL>
__device__ __forceinline__ void view_cols(uint32_t a, uint32_t rs, float f, float4 w,
                                          float2 (&acc)[(RPL + 1) / 2][2 * H][C]) {
    if constexpr (RPL % 2 == 0) {
        const float2 f2 = make_float2(f, f);
        float2 w2[2 * H];
        w2[0] = make_float2(w.x, w.x);
        w2[1] = make_float2(w.y, w.y);
        if constexpr (H == 2) {
            w2[2] = make_float2(w.z, w.z);
            w2[3] = make_float2(w.w, w.w);
        }
#pragma unroll
        for (int rp = 0; rp < RPL / 2; ++rp) {
            const uint32_t ar = a + rs * (uint32_t)(2 * rp);
            row_pair_cols<TQ, C, H>(ar, ar + rs, f2, w2, acc[rp], std::make_integer_sequence<int, C>{});
        }
    } else {
        static_assert(RPL == 1, "an odd number of rows per lane is one row");
        row_cols<TQ, C, H>(a, f, w, acc[0], std::make_integer_sequence<int, C>{});
    }
}

template <typename TQ, int C, int H, int RPL>
__global__ void __launch_bounds__(kDecThreads)
decompose_tma_kernel(const __grid_constant__ CUtensorMap tmap, float *__restrict__ Sp,
                     const int32_t *__restrict__ crop, const GeomEntry *__restrict__ geo,
                     const int32_t *__restrict__ Tq, const float4 *__restrict__ tapw, int *status, int Tstride, int P,
                     int D, int Pd, int Nv, int Wc, int tile_stride, int rowoff, int rowend) {
    constexpr int ES = (int)sizeof(TQ);
    constexpr int kAlign = 16 / ES;
    constexpr int kG = Ring<TQ>::kG, kStages = Ring<TQ>::kStages;
    constexpr int VB = kConsumerWarps * RPL;   // rows per CTA (box height)
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char *ring = smem_raw + ((128u - (tma::smem_u32(smem_raw) & 127u)) & 127u);
    const uint32_t tile_bytes = (uint32_t)(ES * tile_stride);
    // views streamed: k' = -(H D - 1) .. P - 1 + (H - 1) D (view k' mod P)
    const int nstream = P + (2 * H - 1) * D - 1;
    const int nstage = (nstream + kG - 1) / kG;
    float4 *s_taps = (float4 *)(ring + (size_t)tile_bytes * kStages * kG + kColSlack(C));
    float2 *s_fc = (float2 *)(s_taps + D);
    int *s_c = (int *)(s_fc + nstream);
    __shared__ __align__(8) uint64_t full[kStages], empty[kStages];

    const int q = blockIdx.x;
    const int v0 = rowoff + blockIdx.y * VB;
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

    const int rib = ty * RPL;  // first of the warp's rows in the band
    const int v = v0 + rib;
    const int T = Tq[q];
    constexpr int RP = (RPL + 1) / 2;  // row pairs
    float2 acc[RP][2 * H][C];
#pragma unroll
    for (int r = 0; r < RP; ++r)
#pragma unroll
        for (int m = 0; m < 2 * H; ++m)
#pragma unroll
            for (int i = 0; i < C; ++i) acc[r][m][i] = make_float2(0.f, 0.f);
    const size_t vstride = (size_t)Nv * Tstride;
    float *out = Sp + ((size_t)q * Pd * Nv + v) * Tstride + tx;  // row v; row v + r is r Tstride further
    const uint32_t lane_addr = tma::smem_u32(ring) + (uint32_t)(ES * (rib * Wc + tx));
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
                view_cols<TQ, C, H, RPL>(sa + tile_bytes * (uint32_t)w + (uint32_t)(ES * (code & (kAlign - 1))),
                                         row_bytes, fc.x, tp, acc);
                if (code & kCodeRotate) {
                    const int jst = (code >> kCodeStoreShift) - 1;
                    if (jst >= 0) {
#pragma unroll
                        for (int r = 0; r < RPL; ++r) {
                            if (v + r < rowend) {
                                float *dst = out + (size_t)jst * vstride + (size_t)r * Tstride;
#pragma unroll
                                for (int i = 0; i < C; ++i) {
                                    const float val = (r & 1) ? acc[r / 2][0][i].y : acc[r / 2][0][i].x;
                                    if (tx + 32 * i < Tstride) dst[32 * i] = tx + 32 * i < T ? val : 0.f;
                                }
                            }
                        }
                    }
#pragma unroll
                    for (int r = 0; r < RP; ++r)
#pragma unroll
                        for (int i = 0; i < C; ++i) {
#pragma unroll
                            for (int m = 0; m < 2 * H - 1; ++m) acc[r][m][i] = acc[r][m + 1][i];
                            acc[r][2 * H - 1][i] = make_float2(0.f, 0.f);
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

// columns per lane C (lane t takes t, t + 32, ...) from the decomposed row length
inline int dec_cols(int Tstride) { return Tstride <= 32 ? 1 : Tstride <= 64 ? 2 : Tstride <= 128 ? 4 : 8; }

// Rows of a launch: the arrays hold `layout` rows per view (S' included)
// and the launch covers rows rowoff .. rowend - 1 of them.
struct Rows {
    int layout, rowoff, rowend;
};

template <typename TQ, int C, int H, int RPL>
cudaError_t launch_tma_shape(const PlanImpl &p, const CUtensorMap &map, float *out, int Wc, cudaStream_t st,
                             Rows rw, size_t smem, int tile_stride) {
    cudaError_t e = ensure_smem<decompose_tma_kernel<TQ, C, H, RPL>>(smem);
    if (e != cudaSuccess) return e;
    constexpr int VB = kConsumerWarps * RPL;
    dim3 grid(p.od.nsq, (rw.rowend - rw.rowoff + VB - 1) / VB);
    decompose_tma_kernel<TQ, C, H, RPL><<<grid, kDecThreads, smem, st>>>(
        map, out, p.od.crop, p.od.geo, p.od.T, p.tapw, p.status, p.Tstride, p.g.P, p.D, p.Pd, rw.layout, Wc,
        tile_stride, rw.rowoff, rw.rowend);
    return cudaGetLastError();
}

template <typename TQ, int H, int RPL>
cudaError_t launch_tma_c(const PlanImpl &p, const CUtensorMap &map, float *out, int Wc, cudaStream_t st, Rows rw,
                         size_t smem, int tile_stride) {
    switch (dec_cols(p.Tstride)) {
        case 1: return launch_tma_shape<TQ, 1, H, RPL>(p, map, out, Wc, st, rw, smem, tile_stride);
        case 2: return launch_tma_shape<TQ, 2, H, RPL>(p, map, out, Wc, st, rw, smem, tile_stride);
        case 4: return launch_tma_shape<TQ, 4, H, RPL>(p, map, out, Wc, st, rw, smem, tile_stride);
        default: return launch_tma_shape<TQ, 8, H, RPL>(p, map, out, Wc, st, rw, smem, tile_stride);
    }
}

template <typename TQ, int H>
cudaError_t launch_tma_h(const PlanImpl &p, const CUtensorMap &map, float *out, int Wc, cudaStream_t st, Rows rw,
                         size_t smem, int tile_stride, bool wide) {
    return wide ? launch_tma_c<TQ, H, rows_per_lane(H, true)>(p, map, out, Wc, st, rw, smem, tile_stride)
                : launch_tma_c<TQ, H, rows_per_lane(H, false)>(p, map, out, Wc, st, rw, smem, tile_stride);
}

// the wide rows-per-lane shape unless its grid would not fill two waves
bool wide_rows(const PlanImpl &p, int H, int nrows) {
    int dev = 0, sms = 148;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int vb = kConsumerWarps * rows_per_lane(H, true);
    return (long long)p.od.nsq * ((nrows + vb - 1) / vb) >= 2LL * sms;
}

// TMA applies when Q's rows are whole 16-byte units, Q and S' are 16-byte
// aligned (vector stores), a crop box (T_max + one interpolation neighbour +
// alignment) fits 256 columns, D <= 128 and the ring plus the stream tables
// fit in shared memory.
template <typename TQ>
cudaError_t try_tma(const PlanImpl &p, const TQ *Q, float *out, cudaStream_t st, Rows rw, bool &launched) {
    const int nrows = rw.layout;
    launched = false;
    constexpr int kAlign = 16 / (int)sizeof(TQ);
    if ((p.g.Nu % kAlign) != 0 || ((uintptr_t)Q & 15) != 0 || ((uintptr_t)out & 15) != 0) return cudaSuccess;
    const int Wc = (p.od.Tmax + 1 + (kAlign - 1) + (kAlign - 1)) & ~(kAlign - 1);
    if (Wc > 256 || p.Tstride > 256 || p.D > kMaxTapD) return cudaSuccess;  // block offset: 8 bits of the code
    const bool wide = wide_rows(p, p.tap_blocks, rw.rowend - rw.rowoff);
    const int VB = kConsumerWarps * rows_per_lane(p.tap_blocks, wide);
    const int tile_stride = (VB * Wc + 63) & ~63;  // elements; 128-byte multiple for every type
    const int nstream = p.g.P + (2 * p.tap_blocks - 1) * p.D - 1;
    const size_t smem = 128 + sizeof(TQ) * (size_t)Ring<TQ>::kStages * Ring<TQ>::kG * tile_stride +
                        kColSlack(dec_cols(p.Tstride)) +
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
    if (p.tap_blocks == 2) return launch_tma_h<TQ, 2>(p, map, out, Wc, st, rw, smem, tile_stride, wide);
    return launch_tma_h<TQ, 1>(p, map, out, Wc, st, rw, smem, tile_stride, wide);
}

template <typename TQ>
cudaError_t launch_t(const PlanImpl &p, const TQ *Q, float *out, cudaStream_t st, Rows rw) {
    if (p.tap_blocks != 1 && p.tap_blocks != 2) return cudaErrorInvalidValue;
    bool launched = false;
    cudaError_t te = try_tma(p, Q, out, st, rw, launched);
    if (launched || te != cudaSuccess) return te;
    dim3 grid((p.Tstride + kTX - 1) / kTX, (rw.rowend - rw.rowoff + kTY - 1) / kTY, p.od.nsq);
    if (p.tap_blocks == 2)
        decompose_kernel<TQ, 2><<<grid, dim3(kTX, kTY), 0, st>>>(Q, out, p.od.crop, p.od.geo, p.od.T, p.tapw,
                                                                 p.Tstride, p.g.P, p.D, p.Pd, rw.layout, p.g.Nu,
                                                                 rw.rowoff, rw.rowend);
    else
        decompose_kernel<TQ, 1><<<grid, dim3(kTX, kTY), 0, st>>>(Q, out, p.od.crop, p.od.geo, p.od.T, p.tapw,
                                                                 p.Tstride, p.g.P, p.D, p.Pd, rw.layout, p.g.Nu,
                                                                 rw.rowoff, rw.rowend);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_decompose(const PlanImpl &p, const void *Q, float *out, cudaStream_t st, Band b) {
    const int nrows = b.nrows < 0 ? p.g.Nv : b.nrows;
    Rows rw{nrows, 0, nrows};
    if (b.whole_arrays) rw = Rows{p.g.Nv, b.row0, b.row0 + nrows};
    if (p.net) {
        if (b.whole_arrays && (b.row0 != 0 || nrows != p.g.Nv)) return cudaErrorInvalidValue;
        return launch_net_decompose(p, Q, out, st, nrows);
    }
    switch (p.qtype) {
        case FDKOD_F32: return launch_t(p, (const float *)Q, out, st, rw);
        case FDKOD_BF16: return launch_t(p, (const __nv_bfloat16 *)Q, out, st, rw);
        case FDKOD_F16: return launch_t(p, (const __half *)Q, out, st, rw);
    }
    return cudaErrorInvalidValue;
}

}  // namespace fdkod
