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

#include "fdkod_internal.cuh"

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

template <typename TQ>
cudaError_t launch_t(const PlanImpl &p, const TQ *Q, float *out, cudaStream_t st) {
    dim3 grid((p.Tstride + kTX - 1) / kTX, (p.g.Nv + kTY - 1) / kTY, p.od.nsq);
    decompose_kernel<TQ><<<grid, dim3(kTX, kTY), 0, st>>>(Q, out, p.od.crop, p.od.geo, p.od.T, p.Tstride, p.g.P,
                                                          p.D, p.Pd, p.g.Nv, p.g.Nu);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_decompose(const PlanImpl &p, const void *Q, float *out, cudaStream_t st) {
    switch (p.qtype) {
        case FDKOD_F32: return launch_t(p, (const float *)Q, out, st);
        case FDKOD_BF16: return launch_t(p, (const __nv_bfloat16 *)Q, out, st);
        case FDKOD_F16: return launch_t(p, (const __half *)Q, out, st);
    }
    return cudaErrorInvalidValue;
}

}  // namespace fdkod
