// Decomposition stage of FDK-OD (Sec. 2.1): for every square q, detector row
// v and shifted column t, shift each view's row so the square centre sits
// on one column (linear interpolation at column phi_k + w0 + t, i.e. crop
// column c_qk + t with sub-pixel part f_qk), low-pass it along the view
// axis with the triangle taps (D - |i|) / D^2 (circular over the orbit) and
// keep every D-th view.  One thread owns one (q, v, t) and streams the P
// views in order: view k = jD + r adds (D - r) / D^2 of its sample to
// decimated view j and r / D^2 to view j + 1, so only two running sums are
// live.  Consecutive threads take consecutive t, so each view's crop row
// is read as one coalesced segment; CTAs of all squares for the same rows
// run together and share those rows through L2.
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

template <typename TQ>
__global__ void __launch_bounds__(kTX *kTY)
decompose_kernel(const TQ *__restrict__ Q, float *__restrict__ Sp, const int32_t *__restrict__ crop,
                 const GeomEntry *__restrict__ geo, const int32_t *__restrict__ Tq, int Tstride, int P, int D,
                 int Pd, int Nv, int Nu) {
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
    const float inv = 1.0f / (float)(D * D);
    // the last block of views feeds decimated view 0 (circular orbit)
    float cur = 0.f, nxt = 0.f;
    for (int r = 1; r < D; ++r) cur = fmaf((float)r, sample((Pd - 1) * D + r), cur);
    for (int j = 0; j < Pd; ++j) {
        for (int r = 0; r < D; ++r) {
            const float sm = sample(j * D + r);
            cur = fmaf((float)(D - r), sm, cur);
            nxt = fmaf((float)r, sm, nxt);
        }
        out[(size_t)j * vstride] = cur * inv;
        cur = nxt;
        nxt = 0.f;
    }
}


// ---------------------------------------------------------------------------
// TMA path: one CTA per (square q, band of VB detector rows), warp
// specialised.  The producer warp's lane 0 brings each view's crop box
// (VB rows x Wc columns starting at the 16-byte aligned column below
// crop[q][k]) into a ring of kStages slots of kG views with 3D bulk-tensor
// copies (zero fill outside the detector); slot n is full when its bytes
// have landed (mbarrier full[n]) and free again when all consumer warps
// have arrived on empty[n].  No block-wide barrier inside the view loop.
//
// Consumers: LPR lanes share a detector row and each lane owns C
// consecutive columns t0 .. t0 + C - 1, so one view costs the lane a few
// vector shared loads at compile-time offsets (the column offset of the
// crop inside its aligned box selects one of four code paths, uniform per
// view) and, per column, one lerp and the two tap FMAs.  Everything else
// a view needs -- shift fraction, which triangle taps apply and whether a
// decimated view is complete -- is one 8-byte entry of a per-CTA table in
// stream order, built once from crop[q][.] and frac[q][.].

constexpr int kConsumerWarps = 8, kG = 4, kStages = 3;
constexpr int kDecThreads = 32 * (kConsumerWarps + 1);
constexpr int kRingSlack = 128;  // bytes after the ring: vector loads of the last row may run past its end
constexpr uint64_t kDecWaitNs = 2000000000ull;

// code word of a table entry: bits 0-2 the crop's offset inside its aligned
// box, bit 3 "last view of a decimated block" (rotate the running sums),
// bits 4-11 the tap pair, bits 12.. the decimated view to store plus one
// (0: none, the wrapped block).  D <= 128, so 2D tap pairs fit 8 bits.
constexpr int kCodeRotate = 8, kCodeTapShift = 4, kCodeStoreShift = 12;

// Per-CTA tables over the stream positions pos = 0 .. P + D - 2 (view
// k' = pos - (D - 1), taken mod P): s_fc[pos] = {shift fraction of square q,
// code word}, s_c[pos] = crop column, and the 2D tap pairs s_taps[r] =
// (D - r, r) and, for the wrapped block, s_taps[D + r] = (0, r).
template <int kAl>
__device__ __forceinline__ void build_stream_table(float2 *s_fc, int *s_c, float2 *s_taps,
                                                   const int32_t *__restrict__ crop,
                                                   const GeomEntry *__restrict__ geo, int q, int P, int D) {
    const int nstream = P + D - 1;
    for (int pos = threadIdx.x; pos < nstream; pos += blockDim.x) {
        const int kp = pos - (D - 1);
        const int kk = kp < 0 ? kp + P : kp;
        const int c = crop[(size_t)q * P + kk];
        int j, r;
        if (kp < 0) {
            j = -1;
            r = kp + D;
        } else {
            j = kp / D;
            r = kp - j * D;
        }
        int code = (c & (kAl - 1)) | ((j < 0 ? D + r : r) << kCodeTapShift);
        if (r == D - 1) code |= kCodeRotate | ((j + 1) << kCodeStoreShift);
        s_fc[pos] = make_float2(geo[(size_t)q * P + kk].frac, __int_as_float(code));
        s_c[pos] = c;
    }
    for (int i = threadIdx.x; i < 2 * D; i += blockDim.x)
        s_taps[i] = i < D ? make_float2((float)(D - i), (float)i) : make_float2(0.f, (float)(i - D));
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

// One view for one lane: columns t0 + i (i < C) sample the row at box column
// O + i (+ the shift fraction f) and feed the two running sums.
template <typename TQ, int C, int O>
__device__ __forceinline__ void view_cols(uint32_t a, float f, float wa, float wb, float *cur, float *nxt) {
    constexpr int NV = (O + C) / 4 + 1;  // vectors covering elements O .. O + C
    float e[4 * NV];
    VecLoad<TQ, NV>::f(a, e);
#pragma unroll
    for (int i = 0; i < C; ++i) {
        const float a0 = e[O + i], a1 = e[O + i + 1];
        const float smp = fmaf(f, a1 - a0, a0);
        cur[i] = fmaf(wa, smp, cur[i]);
        nxt[i] = fmaf(wb, smp, nxt[i]);
    }
}

// off: the crop's offset inside its 16-byte aligned box (elements).  For
// 16-bit data the vectors are 8 bytes, so the lane's address moves by whole
// vectors and the remainder (0..3) picks the code path.
template <typename TQ, int C>
__device__ __forceinline__ void view_step(uint32_t a, int off, float f, float wa, float wb, float *cur, float *nxt) {
    if (sizeof(TQ) == 2) a += 8u * (uint32_t)(off >> 2);
    switch (off & 3) {
        case 0: view_cols<TQ, C, 0>(a, f, wa, wb, cur, nxt); break;
        case 1: view_cols<TQ, C, 1>(a, f, wa, wb, cur, nxt); break;
        case 2: view_cols<TQ, C, 2>(a, f, wa, wb, cur, nxt); break;
        default: view_cols<TQ, C, 3>(a, f, wa, wb, cur, nxt); break;
    }
}

template <typename TQ, int C, int LPR>
__global__ void __launch_bounds__(kDecThreads)
decompose_tma_kernel(const __grid_constant__ CUtensorMap tmap, float *__restrict__ Sp,
                     const int32_t *__restrict__ crop, const GeomEntry *__restrict__ geo,
                     const int32_t *__restrict__ Tq, int *status, int Tstride, int P, int D, int Pd, int Nv, int Wc,
                     int tile_stride) {
    constexpr int ES = (int)sizeof(TQ);
    constexpr int kAlign = 16 / ES;
    constexpr int RPW = 32 / LPR;              // detector rows per consumer warp
    constexpr int VB = kConsumerWarps * RPW;   // rows per CTA (box height)
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char *ring = smem_raw + ((128u - (tma::smem_u32(smem_raw) & 127u)) & 127u);
    const uint32_t tile_bytes = (uint32_t)(ES * tile_stride);
    // views streamed: k' = -(D-1) .. P-1 (view k' mod P); the first D-1
    // (the orbit's last block) only seed decimated view 0
    const int nstream = P + D - 1;
    const int nstage = (nstream + kG - 1) / kG;
    float2 *s_fc = (float2 *)(ring + (size_t)tile_bytes * kStages * kG + kRingSlack);
    float2 *s_taps = s_fc + nstream;
    int *s_c = (int *)(s_taps + 2 * D);
    __shared__ __align__(8) uint64_t full[kStages], empty[kStages];

    const int q = blockIdx.x;
    const int v0 = blockIdx.y * VB;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;

    build_stream_table<kAlign>(s_fc, s_c, s_taps, crop, geo, q, P, D);
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
        int kk = D > 1 ? P - (D - 1) : 0, n = 0, slot = 0;
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

    const int rib = ty * RPW + tx / LPR;  // row in the band
    const int t0 = (tx % LPR) * C;        // first column of the lane
    const int v = v0 + rib;
    const int T = Tq[q];
    const bool act = t0 < T;
    const bool store = v < Nv && t0 < Tstride;
    float cur[C], nxt[C];
#pragma unroll
    for (int i = 0; i < C; ++i) cur[i] = nxt[i] = 0.f;
    const float inv = 1.0f / (float)(D * D);
    const size_t vstride = (size_t)Nv * Tstride;
    float *out = Sp + ((size_t)q * Pd * Nv + v) * Tstride + t0;
    const uint32_t lane_addr = tma::smem_u32(ring) + (uint32_t)(ES * (rib * Wc + t0));
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
                const float2 tp = s_taps[(code >> kCodeTapShift) & 255];
                if (act) view_step<TQ, C>(sa + tile_bytes * (uint32_t)w, code & (kAlign - 1), fc.x, tp.x, tp.y, cur, nxt);
                if (code & kCodeRotate) {
                    const int jst = (code >> kCodeStoreShift) - 1;
                    if (jst >= 0 && store) {
                        float o[C];
#pragma unroll
                        for (int i = 0; i < C; ++i) o[i] = t0 + i < T ? cur[i] * inv : 0.f;
                        float4 *dst = (float4 *)(out + (size_t)jst * vstride);
#pragma unroll
                        for (int i = 0; i < C / 4; ++i)  // Tstride is a multiple of 4
                            if (t0 + 4 * i < Tstride) dst[i] = make_float4(o[4 * i], o[4 * i + 1], o[4 * i + 2], o[4 * i + 3]);
                    }
#pragma unroll
                    for (int i = 0; i < C; ++i) {
                        cur[i] = nxt[i];
                        nxt[i] = 0.f;
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

template <typename TQ, int C, int LPR>
cudaError_t launch_tma_shape(const PlanImpl &p, const CUtensorMap &map, float *out, int Wc, cudaStream_t st,
                             int nrows, size_t smem, int tile_stride) {
    cudaError_t e = ensure_smem<decompose_tma_kernel<TQ, C, LPR>>(smem);
    if (e != cudaSuccess) return e;
    constexpr int VB = kConsumerWarps * (32 / LPR);
    dim3 grid(p.od.nsq, (nrows + VB - 1) / VB);
    decompose_tma_kernel<TQ, C, LPR><<<grid, kDecThreads, smem, st>>>(map, out, p.od.crop, p.od.geo, p.od.T,
                                                                      p.status, p.Tstride, p.g.P, p.D, p.Pd, nrows,
                                                                      Wc, tile_stride);
    return cudaGetLastError();
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
    if (Wc > 256 || p.Tstride > 256 || p.D > 128) return cudaSuccess;  // tap pair index: 8 bits
    const DecShape sh = dec_shape(p.Tstride);
    const int VB = kConsumerWarps * (32 / sh.LPR);
    const int tile_stride = (VB * Wc + 63) & ~63;  // elements; 128-byte multiple for every type
    const size_t smem = 128 + sizeof(TQ) * (size_t)kStages * kG * tile_stride + kRingSlack +
                        12 * (size_t)(p.g.P + p.D - 1) + 16 * (size_t)p.D;
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
    if (sh.C == 8) return launch_tma_shape<TQ, 8, 32>(p, map, out, Wc, st, nrows, smem, tile_stride);
    if (sh.LPR == 32) return launch_tma_shape<TQ, 4, 32>(p, map, out, Wc, st, nrows, smem, tile_stride);
    if (sh.LPR == 16) return launch_tma_shape<TQ, 4, 16>(p, map, out, Wc, st, nrows, smem, tile_stride);
    return launch_tma_shape<TQ, 4, 8>(p, map, out, Wc, st, nrows, smem, tile_stride);
}

template <typename TQ>
cudaError_t launch_t(const PlanImpl &p, const TQ *Q, float *out, cudaStream_t st, int nrows) {
    bool launched = false;
    cudaError_t te = try_tma(p, Q, out, st, nrows, launched);
    if (launched || te != cudaSuccess) return te;
    dim3 grid((p.Tstride + kTX - 1) / kTX, (nrows + kTY - 1) / kTY, p.od.nsq);
    decompose_kernel<TQ><<<grid, dim3(kTX, kTY), 0, st>>>(Q, out, p.od.crop, p.od.geo, p.od.T, p.Tstride, p.g.P,
                                                          p.D, p.Pd, nrows, p.g.Nu);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_decompose(const PlanImpl &p, const void *Q, float *out, cudaStream_t st, Band b) {
    const int nrows = b.nrows < 0 ? p.g.Nv : b.nrows;
    switch (p.qtype) {
        case FDKOD_F32: return launch_t(p, (const float *)Q, out, st, nrows);
        case FDKOD_BF16: return launch_t(p, (const __nv_bfloat16 *)Q, out, st, nrows);
        case FDKOD_F16: return launch_t(p, (const __half *)Q, out, st, nrows);
    }
    return cudaErrorInvalidValue;
}

}  // namespace fdkod
