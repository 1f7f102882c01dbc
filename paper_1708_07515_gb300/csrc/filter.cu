// FDK filter stage (Sec. 1; the "initial convolution" of Sec. 3): cosine
// weight, then linear convolution of every detector row with the discrete
// Ram-Lak kernel, done as a zero-padded FFT convolution of length
// L >= 2 Nu in shared memory.  Two rows share one complex transform (row A
// in the real part, row B in the imaginary part); the kernel's spectrum is
// real and even, so after the pointwise product the inverse transform
// returns filtered A in the real part and filtered B in the imaginary part.
// The transforms are radix-4 Stockham passes (plus one radix-2 pass when
// log2 L is odd) between two shared-memory buffers, one CTA of L/4 threads
// per row pair; the twiddle table holds e^{-2 pi i m / L} for m < L.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>

#include "fdkod_internal.cuh"

namespace fdkod {
namespace {

constexpr int kThreads = 1024;

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

// One Stockham pass (natural-order input and output, ping-pong buffers):
// item j reads R samples j + r L/R, twiddles them by e^{-2 pi i r (j mod Ns) / (Ns R)},
// does an R-point DFT and writes them to (j / Ns) Ns R + (j mod Ns) + r Ns.
template <int R>
__device__ __forceinline__ void stockham_pass(const float2 *__restrict__ in, float2 *__restrict__ out,
                                              const float2 *__restrict__ tw, int L, int Ns) {
    const int n_items = L / R;
    const int tstep = L / (Ns * R);
    for (int j = threadIdx.x; j < n_items; j += blockDim.x) {
        const int k = j % Ns;
        float2 v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = in[j + r * n_items];
#pragma unroll
        for (int r = 1; r < R; ++r) v[r] = cmul(v[r], tw[r * k * tstep]);
        if (R == 4) {
            const float2 s02 = make_float2(v[0].x + v[2].x, v[0].y + v[2].y);
            const float2 d02 = make_float2(v[0].x - v[2].x, v[0].y - v[2].y);
            const float2 s13 = make_float2(v[1].x + v[3].x, v[1].y + v[3].y);
            const float2 d13 = make_float2(v[1].x - v[3].x, v[1].y - v[3].y);
            v[0] = make_float2(s02.x + s13.x, s02.y + s13.y);
            v[2] = make_float2(s02.x - s13.x, s02.y - s13.y);
            // -i * d13 = (d13.y, -d13.x)
            v[1] = make_float2(d02.x + d13.y, d02.y - d13.x);
            v[3] = make_float2(d02.x - d13.y, d02.y + d13.x);
        } else {
            const float2 a = v[0], b = v[1];
            v[0] = make_float2(a.x + b.x, a.y + b.y);
            v[1] = make_float2(a.x - b.x, a.y - b.y);
        }
        const int d = (j - k) * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) out[d + r * Ns] = v[r];
    }
}

// Forward DFT of length L = 2^log2L held in a; returns the buffer holding
// the result (a or b).
__device__ __forceinline__ float2 *fft_forward(float2 *a, float2 *b, const float2 *tw, int L, int log2L) {
    int Ns = 1;
    for (int p = 0; p + 2 <= log2L; p += 2) {
        stockham_pass<4>(a, b, tw, L, Ns);
        __syncthreads();
        float2 *t = a;
        a = b;
        b = t;
        Ns *= 4;
    }
    if (log2L & 1) {
        stockham_pass<2>(a, b, tw, L, Ns);
        __syncthreads();
        float2 *t = a;
        a = b;
        b = t;
    }
    return a;
}

template <typename TQ>
__global__ void __launch_bounds__(kThreads)
filter_kernel(const float *__restrict__ proj, TQ *__restrict__ Q, const float *__restrict__ H,
              const float2 *__restrict__ tw, int L, int log2L, int Nu, int Nv, long long nrows, float R) {
    extern __shared__ float2 z[];
    float2 *a = z, *b = z + L;
    const long long rowA = 2LL * blockIdx.x;
    const long long rowB = rowA + 1;
    const bool hasB = rowB < nrows;
    const float *pA = proj + rowA * Nu;
    const float *pB = proj + rowB * Nu;
    const float bA = (float)(rowA % Nv) - 0.5f * (float)(Nv - 1);
    const float bB = (float)(rowB % Nv) - 0.5f * (float)(Nv - 1);
    const float R2 = R * R;
    for (int i = threadIdx.x; i < L; i += blockDim.x) {
        float2 v = make_float2(0.f, 0.f);
        if (i < Nu) {
            const float u = (float)i - 0.5f * (float)(Nu - 1);
            v.x = __ldg(pA + i) * (R / sqrtf(R2 + u * u + bA * bA));
            if (hasB) v.y = __ldg(pB + i) * (R / sqrtf(R2 + u * u + bB * bB));
        }
        a[i] = v;
    }
    __syncthreads();
    float2 *x = fft_forward(a, b, tw, L, log2L);
    // product with the real, even ramp spectrum (1/L folded in), conjugated:
    // the inverse transform is the conjugate of a forward transform
    for (int i = threadIdx.x; i < L; i += blockDim.x) {
        const float h = H[i];
        const float2 v = x[i];
        x[i] = make_float2(v.x * h, -v.y * h);
    }
    __syncthreads();
    float2 *y = fft_forward(x, x == a ? b : a, tw, L, log2L);
    TQ *qA = Q + rowA * Nu;
    TQ *qB = Q + rowB * Nu;
    for (int u = threadIdx.x; u < Nu; u += blockDim.x) {
        const float2 v = y[u];
        qA[u] = to_q<TQ>(v.x);
        if (hasB) qB[u] = to_q<TQ>(-v.y);
    }
}

template <typename TQ>
cudaError_t launch_t(const PlanImpl &p, const float *proj, TQ *Q, cudaStream_t st) {
    const long long nrows = (long long)p.g.P * p.g.Nv;
    const long long blocks = (nrows + 1) / 2;
    const size_t smem = 2 * sizeof(float2) * (size_t)p.L;
    cudaError_t e = cudaFuncSetAttribute(filter_kernel<TQ>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    const int threads = std::max(32, std::min(kThreads, p.L / 4));
    filter_kernel<TQ><<<(unsigned)blocks, threads, smem, st>>>(proj, Q, p.H, p.tw, p.L, p.log2L, p.g.Nu,
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
