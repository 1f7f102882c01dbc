// FDK filter stage (Sec. 1; the "initial convolution" of Sec. 3): cosine
// weight, then linear convolution of every detector row with the discrete
// Ram-Lak kernel, done as a zero-padded FFT convolution of length
// L >= 2 Nu in shared memory.  Two rows share one complex transform (row A
// in the real part, row B in the imaginary part); the kernel's spectrum is
// real and even, so after the pointwise product the inverse transform
// returns filtered A in the real part and filtered B in the imaginary part.
// The transforms are in-place Stockham passes of radix 16 (16-point DFTs in
// registers) plus one pass of radix 2, 4 or 8; L/16 threads per row pair and
// several pairs per CTA; the twiddle table holds e^{-2 pi i m / L}, m < L.
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

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
// multiply by -i
__device__ __forceinline__ float2 cmi(float2 a) { return make_float2(a.y, -a.x); }

// 4-point forward DFT in place: (a, b, c, d) -> (X0, X1, X2, X3)
__device__ __forceinline__ void dft4(float2 &a, float2 &b, float2 &c, float2 &d) {
    const float2 s02 = cadd(a, c), d02 = csub(a, c), s13 = cadd(b, d), d13 = csub(b, d);
    a = cadd(s02, s13);
    c = csub(s02, s13);
    b = cadd(d02, cmi(d13));
    d = csub(d02, cmi(d13));
}

constexpr float kC1 = 0.92387953251128674f;  // cos(pi/8)
constexpr float kS1 = 0.38268343236508978f;  // sin(pi/8)
constexpr float kH = 0.70710678118654752f;   // cos(pi/4)

// R-point forward DFT of v in registers; result X[k] left at v[pos(k)]
// with pos(k) = (R/4) (k mod 4) + k / 4 for R = 16 and 2 (k mod 4) + k / 4
// for R = 8 (the 4 x R/4 index map); R = 4, 2: natural order.
template <int R>
__device__ __forceinline__ void dft(float2 *v);

template <>
__device__ __forceinline__ void dft<2>(float2 *v) {
    const float2 a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
}

template <>
__device__ __forceinline__ void dft<4>(float2 *v) { dft4(v[0], v[1], v[2], v[3]); }

template <>
__device__ __forceinline__ void dft<8>(float2 *v) {
    // n = 2 n1 + n2: 4-point DFTs over n1, twiddle W8^(n2 k1), 2-point over n2
    dft4(v[0], v[2], v[4], v[6]);
    dft4(v[1], v[3], v[5], v[7]);
    v[3] = cmul(v[3], make_float2(kH, -kH));
    v[5] = cmi(v[5]);
    v[7] = cmul(v[7], make_float2(-kH, -kH));
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) {
        const float2 a = v[2 * k1], b = v[2 * k1 + 1];
        v[2 * k1] = cadd(a, b);
        v[2 * k1 + 1] = csub(a, b);
    }
}

template <>
__device__ __forceinline__ void dft<16>(float2 *v) {
    // n = 4 n1 + n2: 4-point DFTs over n1, twiddle W16^(n2 k1), 4-point over n2
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) dft4(v[n2], v[4 + n2], v[8 + n2], v[12 + n2]);
    // position n2 + 4 k1 holds Y[n2][k1]
    v[1 + 4 * 1] = cmul(v[1 + 4 * 1], make_float2(kC1, -kS1));   // W16^1
    v[1 + 4 * 2] = cmul(v[1 + 4 * 2], make_float2(kH, -kH));     // W16^2
    v[1 + 4 * 3] = cmul(v[1 + 4 * 3], make_float2(kS1, -kC1));   // W16^3
    v[2 + 4 * 1] = cmul(v[2 + 4 * 1], make_float2(kH, -kH));     // W16^2
    v[2 + 4 * 2] = cmi(v[2 + 4 * 2]);                            // W16^4
    v[2 + 4 * 3] = cmul(v[2 + 4 * 3], make_float2(-kH, -kH));    // W16^6
    v[3 + 4 * 1] = cmul(v[3 + 4 * 1], make_float2(kS1, -kC1));   // W16^3
    v[3 + 4 * 2] = cmul(v[3 + 4 * 2], make_float2(-kH, -kH));    // W16^6
    v[3 + 4 * 3] = cmul(v[3 + 4 * 3], make_float2(-kC1, kS1));   // W16^9
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) dft4(v[4 * k1], v[4 * k1 + 1], v[4 * k1 + 2], v[4 * k1 + 3]);
}

template <int R>
__device__ __forceinline__ constexpr int out_pos(int k) {
    return R == 16 ? 4 * (k % 4) + k / 4 : (R == 8 ? 2 * (k % 4) + k / 4 : k);
}

// shared-memory index with one pad slot per 16 (breaks stride-16 conflicts)
__device__ __forceinline__ int pad(int i) { return i + (i >> 4); }

// Where a pass leaves its output: in shared memory (kToSmem); in shared
// memory times the ramp spectrum and conjugated (kToSpectrum, the last pass
// of the forward transform: the inverse transform is the conjugate of a
// forward one); or, for the first Nu samples, in the two output rows of Q
// (kToQ, the last pass of the inverse transform).
enum PassOut { kToSmem, kToSpectrum, kToQ };

template <typename TQ>
struct Sink {
    const float *H;  // ramp spectrum / L
    TQ *qa, *qb;     // output rows (nullptr: absent)
    int Nu;
};

// One Stockham pass of radix R over a buffer of length L (padded):
// item j reads R samples j + r L/R, twiddles them by
// e^{-2 pi i r (j mod Ns) / (Ns R)}, does an R-point DFT and writes sample
// r to (j - j mod Ns) R + (j mod Ns) + r Ns.  Each thread owns 16/R items
// (16 values), all loaded before the barrier that precedes in-place stores.
// L, Ns and L/R are powers of two, so j mod Ns is a mask and the twiddle
// index a shift; when the read stride L/R (write stride Ns) is a multiple of
// 16, the padded index of sample r is the padded index of sample 0 plus r
// times the padded stride, one add per sample.  Ns is 1 on the first pass
// (its samples are consecutive within one 16-block) and a multiple of 16
// after it.
// FIRST: the forward transform's first pass (radix 16, Ns = 1), whose inputs
// r >= 8 lie at j + r L/16 >= L/2 >= Nu, in the zero padding: they are
// constant zeros, neither stored by the input stage nor loaded here.
template <int R, int OUT, typename TQ, bool FIRST = false>
__device__ __forceinline__ void pass(float2 *buf, const float2 *__restrict__ tw, int lgL, int lgNs, int lt, int nt,
                                     const Sink<TQ> &sink) {
    constexpr int kItems = 16 / R;
    constexpr int lgR = R == 16 ? 4 : (R == 8 ? 3 : (R == 4 ? 2 : 1));
    const int n_items = 1 << (lgL - lgR);
    const int Ns = 1 << lgNs;
    const int lg_tstep = lgL - lgNs - lgR;
    const bool whole_in = n_items >= 16;       // read stride: whole 16-blocks
    const int pin = n_items + (n_items >> 4);  // its padded length
    const int pout = Ns + (Ns >> 4);           // padded write stride (Ns >= 16)
    float2 v[kItems][R];
    int d0[kItems];
#pragma unroll
    for (int it = 0; it < kItems; ++it) {
        const int j = lt + it * nt;
        const int k = j & (Ns - 1);
        constexpr int kLoad = FIRST ? R / 2 : R;
        if (whole_in) {
            const int b0 = pad(j);
#pragma unroll
            for (int r = 0; r < kLoad; ++r) v[it][r] = buf[b0 + r * pin];
        } else {
#pragma unroll
            for (int r = 0; r < kLoad; ++r) v[it][r] = buf[pad(j + r * n_items)];
        }
#pragma unroll
        for (int r = kLoad; r < R; ++r) v[it][r] = make_float2(0.f, 0.f);
        if (Ns > 1) {
            float2 w[R];
            w[1] = tw[k << lg_tstep];
            if (R >= 4) w[2] = tw[(2 * k) << lg_tstep];
            if (R >= 4) w[3] = cmul(w[1], w[2]);
            if (R >= 8) {
                w[4] = tw[(4 * k) << lg_tstep];
                w[5] = cmul(w[1], w[4]);
                w[6] = cmul(w[2], w[4]);
                w[7] = cmul(w[3], w[4]);
            }
            if (R >= 16) {
                w[8] = tw[(8 * k) << lg_tstep];
#pragma unroll
                for (int r = 9; r < 16; ++r) w[r] = cmul(w[r - 8], w[8]);
            }
#pragma unroll
            for (int r = 1; r < R; ++r) v[it][r] = cmul(v[it][r], w[r]);
        }
        dft<R>(v[it]);
        d0[it] = ((j - k) << lgR) + k;
    }
    if (OUT == kToQ) {
        // natural order after the last pass; only the first Nu samples are kept
#pragma unroll
        for (int it = 0; it < kItems; ++it)
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int i = d0[it] + r * Ns;
                if (i < sink.Nu) {
                    const float2 x = v[it][out_pos<R>(r)];
                    if (sink.qa) sink.qa[i] = to_q<TQ>(x.x);
                    if (sink.qb) sink.qb[i] = to_q<TQ>(-x.y);
                }
            }
        return;
    }
    __syncthreads();
    const int sstride = Ns == 1 ? 1 : pout;  // Ns = 1: R <= 16 consecutive samples of one 16-block
#pragma unroll
    for (int it = 0; it < kItems; ++it) {
        const int dp = pad(d0[it]);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            float2 x = v[it][out_pos<R>(r)];
            if (OUT == kToSpectrum) {
                const float h = __ldg(sink.H + d0[it] + r * Ns);
                x = make_float2(x.x * h, -x.y * h);
            }
            buf[dp + r * sstride] = x;
        }
    }
    __syncthreads();
}

// DFT of length L = 2^log2L (>= 16) in place: radix-16 passes, then one pass
// of radix 2, 4 or 8 for the remaining factor; the last pass writes per OUT.
// The forward transform (OUT = kToSpectrum) starts on data whose upper half
// is zero padding.
template <int OUT, typename TQ>
__device__ __forceinline__ void fft(float2 *buf, const float2 *tw, int lgL, int lt, int nt, const Sink<TQ> &sink) {
    const int rest = lgL & 3;
    const int n16 = lgL >> 2;
    int lgNs = 0;
    for (int p = 0; p < n16; ++p) {
        if (p == n16 - 1 && rest == 0) {
            if (p == 0 && OUT == kToSpectrum) pass<16, OUT, TQ, true>(buf, tw, lgL, lgNs, lt, nt, sink);
            else pass<16, OUT>(buf, tw, lgL, lgNs, lt, nt, sink);
        } else if (p == 0 && OUT == kToSpectrum) {
            pass<16, kToSmem, TQ, true>(buf, tw, lgL, lgNs, lt, nt, sink);
        } else {
            pass<16, kToSmem>(buf, tw, lgL, lgNs, lt, nt, sink);
        }
        lgNs += 4;
    }
    if (rest == 3) pass<8, OUT>(buf, tw, lgL, lgNs, lt, nt, sink);
    else if (rest == 2) pass<4, OUT>(buf, tw, lgL, lgNs, lt, nt, sink);
    else if (rest == 1) pass<2, OUT>(buf, tw, lgL, lgNs, lt, nt, sink);
}

// G row pairs per CTA, L/16 threads per pair: weighted rows into shared
// memory, forward transform (times the spectrum on its last pass), inverse
// transform (its last pass stores the rows of Q).
template <typename TQ>
__global__ void __launch_bounds__(kThreads)
filter_kernel(const float *__restrict__ proj, TQ *__restrict__ Q, const float *__restrict__ H,
              const float2 *__restrict__ tw, int L, int lgL, int G, int Nu, int Nv, int row0, int rows_per_view,
              long long nrows, float R) {
    extern __shared__ float2 z[];
    const int nt = L / 16;
    const int g = threadIdx.x / nt, lt = threadIdx.x % nt;
    float2 *buf = z + (size_t)g * (L + L / 16);
    const long long rowA = 2LL * ((long long)blockIdx.x * G + g);
    const long long rowB = rowA + 1;
    const bool hasA = rowA < nrows, hasB = rowB < nrows;
    // detector row of each input row (the input may hold rows row0 .. of each view)
    const float bA = (float)(row0 + (int)(rowA % rows_per_view)) - 0.5f * (float)(Nv - 1);
    const float bB = (float)(row0 + (int)(rowB % rows_per_view)) - 0.5f * (float)(Nv - 1);
    const float R2 = R * R;
    for (int i = lt; i < L / 2; i += nt) {  // the upper half is never read (see pass)
        float2 v = make_float2(0.f, 0.f);
        if (i < Nu) {
            const float u = (float)i - 0.5f * (float)(Nu - 1);
            if (hasA) v.x = __ldg(proj + rowA * Nu + i) * (R * rsqrtf(R2 + u * u + bA * bA));
            if (hasB) v.y = __ldg(proj + rowB * Nu + i) * (R * rsqrtf(R2 + u * u + bB * bB));
        }
        buf[pad(i)] = v;
    }
    __syncthreads();
    Sink<TQ> sink;
    sink.H = H;
    sink.qa = hasA ? Q + rowA * Nu : nullptr;
    sink.qb = hasB ? Q + rowB * Nu : nullptr;
    sink.Nu = Nu;
    fft<kToSpectrum>(buf, tw, lgL, lt, nt, sink);
    fft<kToQ>(buf, tw, lgL, lt, nt, sink);
}

template <typename TQ>
cudaError_t launch_t(const PlanImpl &p, const float *proj, TQ *Q, cudaStream_t st, int row0, int rows_per_view,
                     int views) {
    const long long nrows = (long long)views * rows_per_view;
    const long long pairs = (nrows + 1) / 2;
    const int G = std::max(1, 2048 / p.L);  // 128 threads per CTA up to L = 2048
    const long long blocks = (pairs + G - 1) / G;
    const size_t smem = sizeof(float2) * (size_t)G * (p.L + p.L / 16);
    cudaError_t e = ensure_smem<filter_kernel<TQ>>(smem);
    if (e != cudaSuccess) return e;
    filter_kernel<TQ><<<(unsigned)blocks, G * (p.L / 16), smem, st>>>(proj, Q, p.H, p.tw, p.L, p.log2L, G, p.g.Nu, p.g.Nv,
                                                                      row0, rows_per_view, nrows, (float)p.g.R);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_filter(const PlanImpl &p, const float *proj, void *Q, cudaStream_t st, Band b, int views) {
    const int rows = b.nrows < 0 ? p.g.Nv : b.nrows;
    if (views < 0) views = p.g.P;
    if (views == 0) return cudaSuccess;
    switch (p.qtype) {
        case FDKOD_F32: return launch_t(p, proj, (float *)Q, st, b.row0, rows, views);
        case FDKOD_BF16: return launch_t(p, proj, (__nv_bfloat16 *)Q, st, b.row0, rows, views);
        case FDKOD_F16: return launch_t(p, proj, (__half *)Q, st, b.row0, rows, views);
    }
    return cudaErrorInvalidValue;
}

}  // namespace fdkod
