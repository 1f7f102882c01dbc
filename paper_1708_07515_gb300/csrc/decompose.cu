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
// TMA path: one CTA per (square q, band of kVB detector rows).  The crop box
// of each view (kVB rows x Wc columns starting at the 16-byte aligned column
// below crop[q][k]) arrives by a 3D bulk-tensor copy, zero-filled outside the
// detector, through a ring of kStages stages of kG views each.  Thread (tx, ty)
// owns row v0 + ty and columns t = tx + 32 i, i < NT, and streams the views
// with two running sums per column as above.

constexpr int kVB = 8, kG = 4, kStages = 4;
constexpr uint64_t kDecWaitNs = 2000000000ull;

template <typename TQ>
__device__ __forceinline__ float sm_ld(const TQ *p);
template <>
__device__ __forceinline__ float sm_ld<float>(const float *p) { return *p; }
template <>
__device__ __forceinline__ float sm_ld<__nv_bfloat16>(const __nv_bfloat16 *p) { return __bfloat162float(*p); }
template <>
__device__ __forceinline__ float sm_ld<__half>(const __half *p) { return __half2float(*p); }

template <typename TQ, int NT>
__global__ void __launch_bounds__(256)
decompose_tma_kernel(const __grid_constant__ CUtensorMap tmap, float *__restrict__ Sp,
                     const int32_t *__restrict__ crop, const GeomEntry *__restrict__ geo,
                     const int32_t *__restrict__ Tq, int *status, int Tstride, int P, int D, int Pd, int Nv, int Wc,
                     int tile_stride) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    TQ *sm = (TQ *)(smem_raw + ((128u - (tma::smem_u32(smem_raw) & 127u)) & 127u));
    // per-view tables after the staging ring
    int *s_crop = (int *)((unsigned char *)sm + sizeof(TQ) * (size_t)kStages * kG * tile_stride);
    float *s_frac = (float *)(s_crop + P);
    __shared__ __align__(8) uint64_t bars[kStages];
    // per view of a stage: shift fraction, column offset in the box, and the
    // triangle-tap weights of its two decimated views (D - r and r, the first
    // zero for the wrapped block), all prepared by the issuing warp
    __shared__ float4 s_vw[kStages][kG];
    __shared__ int s_off[kStages][kG];

    const int q = blockIdx.x;
    const int v0 = blockIdx.y * kVB;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int v = v0 + ty;
    const int T = Tq[q];
    constexpr int kAlign = 16 / (int)sizeof(TQ);
    // views streamed: k' = -(D-1) .. P-1 (view k' mod P)
    const int nstream = P + D - 1;
    const int nstage = (nstream + kG - 1) / kG;

    auto issue = [&](int n) {  // warp 0: views of stage n into slot n % kStages
        const int slot = n % kStages;
        const int base = n * kG;
        const int nv = min(kG, nstream - base);
        int xs = 0, kk = 0;
        if (tx < nv) {
            const int kp = base + tx - (D - 1);
            kk = kp < 0 ? kp + P : kp;
            const int c = s_crop[kk];
            xs = c & ~(kAlign - 1);
            s_off[slot][tx] = c - xs;
            const int r = kp < 0 ? kp + D : kp % D;
            s_vw[slot][tx] = make_float4(s_frac[kk], kp < 0 ? 0.f : (float)(D - r), (float)r, 0.f);
        }
        __syncwarp();
        if (tx == 0) {
            tma::fence_proxy_async();
            tma::mbar_arrive_expect_tx(&bars[slot], (uint32_t)(nv * kVB * Wc * (int)sizeof(TQ)));
        }
        for (int w = 0; w < nv; ++w) {
            const int xw = __shfl_sync(0xffffffffu, xs, w);
            const int kw = __shfl_sync(0xffffffffu, kk, w);
            if (tx == 0)
                tma::load_3d(sm + (size_t)(slot * kG + w) * tile_stride, &tmap, &bars[slot], xw, v0, kw);
        }
    };

    // this square's crop columns and shift fractions, once per CTA
    for (int k = threadIdx.x; k < P; k += blockDim.x) {
        s_crop[k] = crop[(size_t)q * P + k];
        s_frac[k] = geo[(size_t)q * P + k].frac;
    }
    if (threadIdx.x == 0) {
        for (int i = 0; i < kStages; ++i) tma::mbar_init(&bars[i], 1);
        tma::fence_mbar_init();
    }
    __syncthreads();
    if (ty == 0)
        for (int n = 0; n < kStages - 1 && n < nstage; ++n) issue(n);

    float cur[NT], nxt[NT];
#pragma unroll
    for (int i = 0; i < NT; ++i) cur[i] = nxt[i] = 0.f;
    const float inv = 1.0f / (float)(D * D);
    const size_t vstride = (size_t)Nv * Tstride;
    float *out = Sp + ((size_t)q * Pd * Nv + v) * Tstride;
    const bool vok = v < Nv;
    bool valid[NT];
#pragma unroll
    for (int i = 0; i < NT; ++i) valid[i] = tx + 32 * i < T;
    // the stream starts at k' = -(D-1): block j0 = -1, tap r = 1 (D > 1)
    int j0 = D > 1 ? -1 : 0, r = D > 1 ? 1 : 0;

    for (int n = 0; n < nstage; ++n) {
        const int slot = n % kStages;
        if (ty == 0 && n + kStages - 1 < nstage) issue(n + kStages - 1);
        const bool ok = tma::mbar_wait_bounded(&bars[slot], (uint32_t)((n / kStages) & 1), kDecWaitNs);
        if (!__syncthreads_and(ok)) {
            if (threadIdx.x == 0) atomicOr(status, 2);
            for (int m = n; m < nstage && m < n + kStages; ++m)
                tma::mbar_wait_bounded(&bars[m % kStages], (uint32_t)((m / kStages) & 1), kDecWaitNs);
            return;
        }
        const int nv = min(kG, nstream - n * kG);
        for (int w = 0; w < nv; ++w) {
            // stream position -> decimated view j0 (-1 for the wrapped block)
            // and tap r, advanced incrementally (no division)
            const float4 vw = s_vw[slot][w];
            const float f = vw.x, wa = vw.y, wb = vw.z;
                const TQ *row = sm + (size_t)(slot * kG + w) * tile_stride + (size_t)ty * Wc + s_off[slot][w] + tx;
#pragma unroll
                for (int i = 0; i < NT; ++i) {
                    // columns t < T read at most T + 3 < Wc elements into the row
                    if (valid[i]) {
                        const float a0 = sm_ld(row + 32 * i), a1 = sm_ld(row + 32 * i + 1);
                        const float smp = fmaf(f, a1 - a0, a0);
                        cur[i] = fmaf(wa, smp, cur[i]);
                        nxt[i] = fmaf(wb, smp, nxt[i]);
                    }
                }
            if (r == D - 1) {
                if (j0 >= 0 && vok) {
                    float *o = out + (size_t)j0 * vstride;
#pragma unroll
                    for (int i = 0; i < NT; ++i) {
                        const int t = tx + 32 * i;
                        if (t < Tstride) o[t] = t < T ? cur[i] * inv : 0.f;
                    }
                }
                // the wrapped block (j0 = -1) only seeds decimated view 0
#pragma unroll
                for (int i = 0; i < NT; ++i) {
                    cur[i] = nxt[i];
                    nxt[i] = 0.f;
                }
                r = 0;
                ++j0;
            } else {
                ++r;
            }
        }
        __syncthreads();
    }
}

template <typename TQ, int NT>
cudaError_t launch_tma_nt(const PlanImpl &p, const CUtensorMap &map, float *out, int Wc, cudaStream_t st,
                          int nrows) {
    const int tile_stride = (kVB * Wc + 63) & ~63;  // elements; 128-byte multiple for every type
    const size_t smem = sizeof(TQ) * (size_t)kStages * kG * tile_stride + 128 + 8 * (size_t)p.g.P;
    cudaError_t e = ensure_smem<decompose_tma_kernel<TQ, NT>>(smem);
    if (e != cudaSuccess) return e;
    dim3 grid(p.od.nsq, (nrows + kVB - 1) / kVB);
    decompose_tma_kernel<TQ, NT><<<grid, 256, smem, st>>>(map, out, p.od.crop, p.od.geo, p.od.T, p.status, p.Tstride,
                                                          p.g.P, p.D, p.Pd, nrows, Wc, tile_stride);
    return cudaGetLastError();
}

// TMA applies when Q's rows are whole 16-byte units, Q is 16-byte aligned and
// a crop box (T_max + one interpolation neighbour + alignment) fits 256 columns.
template <typename TQ>
cudaError_t try_tma(const PlanImpl &p, const TQ *Q, float *out, cudaStream_t st, int nrows, bool &launched) {
    launched = false;
    constexpr int kAlign = 16 / (int)sizeof(TQ);
    if ((p.g.Nu % kAlign) != 0 || ((uintptr_t)Q & 15) != 0) return cudaSuccess;
    const int Wc = (p.od.Tmax + 1 + (kAlign - 1) + (kAlign - 1)) & ~(kAlign - 1);
    if (Wc > 256 || p.Tstride > 256 || p.g.P > 4096) return cudaSuccess;
    CUtensorMap map;
    const uint64_t dims[3] = {(uint64_t)p.g.Nu, (uint64_t)nrows, (uint64_t)p.g.P};
    const uint64_t strides[2] = {(uint64_t)p.g.Nu * sizeof(TQ), (uint64_t)p.g.Nu * nrows * sizeof(TQ)};
    const uint32_t box[3] = {(uint32_t)Wc, (uint32_t)kVB, 1u};
    const CUtensorMapDataType dt = sizeof(TQ) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                   : (std::is_same<TQ, __half>::value ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                                                      : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16);
    if (encode_map_3d(&map, dt, Q, dims, strides, box) != cudaSuccess) return cudaSuccess;
    launched = true;
    const int nt = (p.Tstride + 31) / 32;
    if (nt <= 2) return launch_tma_nt<TQ, 2>(p, map, out, Wc, st, nrows);
    if (nt <= 4) return launch_tma_nt<TQ, 4>(p, map, out, Wc, st, nrows);
    return launch_tma_nt<TQ, 8>(p, map, out, Wc, st, nrows);
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
