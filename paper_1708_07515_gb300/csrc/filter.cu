// FDK filter stage (Sec. 1; the "initial convolution" of Sec. 3): cosine
// weight, then linear convolution of every detector row with the discrete
// Ram-Lak kernel, done as a zero-padded FFT convolution of length
// L >= 2 Nu in shared memory.  Two rows share one complex transform (row A
// in the real part, row B in the imaginary part); the kernel's spectrum is
// real and even, so after the pointwise product the inverse transform
// returns filtered A in the real part and filtered B in the imaginary part.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "fdkod_internal.cuh"

namespace fdkod {
namespace {

constexpr int kThreads = 512;

template <typename T>
__device__ __forceinline__ T to_q(float x);
template <>
__device__ __forceinline__ float to_q<float>(float x) { return x; }
template <>
__device__ __forceinline__ __nv_bfloat16 to_q<__nv_bfloat16>(float x) { return __float2bfloat16_rn(x); }
template <>
__device__ __forceinline__ __half to_q<__half>(float x) { return __float2half_rn(x); }

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

template <typename TQ>
__global__ void __launch_bounds__(kThreads)
filter_kernel(const float *__restrict__ proj, TQ *__restrict__ Q, const float *__restrict__ H,
              const float2 *__restrict__ tw, int L, int log2L, int Nu, int Nv, long long nrows, float R) {
    extern __shared__ float2 z[];
    const long long rowA = 2LL * blockIdx.x;
    const long long rowB = rowA + 1;
    const bool hasB = rowB < nrows;
    const float *pA = proj + rowA * Nu;
    const float *pB = proj + rowB * Nu;
    const float bA = (float)(rowA % Nv) - 0.5f * (float)(Nv - 1);
    const float bB = (float)(rowB % Nv) - 0.5f * (float)(Nv - 1);
    const float R2 = R * R;
    const int sh = 32 - log2L;
    // weighted rows, loaded in bit-reversed order for the decimation-in-time pass
    for (int i = threadIdx.x; i < L; i += kThreads) {
        float2 v = make_float2(0.f, 0.f);
        if (i < Nu) {
            const float a = (float)i - 0.5f * (float)(Nu - 1);
            v.x = __ldg(pA + i) * (R / sqrtf(R2 + a * a + bA * bA));
            if (hasB) v.y = __ldg(pB + i) * (R / sqrtf(R2 + a * a + bB * bB));
        }
        z[__brev((unsigned)i) >> sh] = v;
    }
    __syncthreads();
    const int half_n = L >> 1;
    // forward transform, decimation in time: natural-order output
    for (int half = 1, tstep = half_n; half < L; half <<= 1, tstep >>= 1) {
        for (int b = threadIdx.x; b < half_n; b += kThreads) {
            const int pos = b & (half - 1);
            const int i = ((b - pos) << 1) + pos;
            const int j = i + half;
            const float2 t = cmul(tw[pos * tstep], z[j]);
            const float2 a = z[i];
            z[i] = make_float2(a.x + t.x, a.y + t.y);
            z[j] = make_float2(a.x - t.x, a.y - t.y);
        }
        __syncthreads();
    }
    // pointwise product with the (real, even) ramp spectrum, 1/L folded in
    for (int i = threadIdx.x; i < L; i += kThreads) {
        const float h = H[i];
        const float2 v = z[i];
        z[i] = make_float2(v.x * h, v.y * h);
    }
    __syncthreads();
    // inverse transform, decimation in frequency: bit-reversed output
    for (int half = half_n, tstep = 1; half >= 1; half >>= 1, tstep <<= 1) {
        for (int b = threadIdx.x; b < half_n; b += kThreads) {
            const int pos = b & (half - 1);
            const int i = ((b - pos) << 1) + pos;
            const int j = i + half;
            const float2 a = z[i], c = z[j];
            const float2 w = tw[pos * tstep];
            z[i] = make_float2(a.x + c.x, a.y + c.y);
            z[j] = cmul(make_float2(a.x - c.x, a.y - c.y), make_float2(w.x, -w.y));
        }
        __syncthreads();
    }
    TQ *qA = Q + rowA * Nu;
    TQ *qB = Q + rowB * Nu;
    for (int u = threadIdx.x; u < Nu; u += kThreads) {
        const float2 v = z[__brev((unsigned)u) >> sh];
        qA[u] = to_q<TQ>(v.x);
        if (hasB) qB[u] = to_q<TQ>(v.y);
    }
}

template <typename TQ>
cudaError_t launch_t(const PlanImpl &p, const float *proj, TQ *Q, cudaStream_t st) {
    const long long nrows = (long long)p.g.P * p.g.Nv;
    const long long blocks = (nrows + 1) / 2;
    const size_t smem = sizeof(float2) * (size_t)p.L;
    cudaError_t e = cudaFuncSetAttribute(filter_kernel<TQ>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    filter_kernel<TQ><<<(unsigned)blocks, kThreads, smem, st>>>(proj, Q, p.H, p.tw, p.L, p.log2L, p.g.Nu,
                                                                p.g.Nv, nrows, (float)p.g.R);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_filter(const PlanImpl &p, const float *proj, void *Q, cudaStream_t st) {
    switch (p.qtype) {
        case FDKOD_F32: return launch_t(p, proj, (float *)Q, st);
        case FDKOD_BF16: return launch_t(p, proj, (__nv_bfloat16 *)Q, st);
        case FDKOD_F16: return launch_t(p, proj, (__half *)Q, st);
    }
    return cudaErrorInvalidValue;
}

}  // namespace fdkod
