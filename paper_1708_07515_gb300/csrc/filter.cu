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
#include "packed.cuh"
#include "tma.cuh"

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

// Complex sum and difference as packed two-lane FP32 instructions (real and
// imaginary part in one instruction, each rounded as the scalar operation
// would be).
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return fsub2(a, b); }
// multiply by -i
__device__ __forceinline__ float2 cmi(float2 a) { return make_float2(a.y, -a.x); }
// a - i d and a + i d (scalar: the swapped operand would cost a move)
__device__ __forceinline__ float2 cadd_mi(float2 a, float2 d) { return make_float2(a.x + d.y, a.y - d.x); }
__device__ __forceinline__ float2 csub_mi(float2 a, float2 d) { return make_float2(a.x - d.y, a.y + d.x); }

// 4-point forward DFT in place: (a, b, c, d) -> (X0, X1, X2, X3)
__device__ __forceinline__ void dft4(float2 &a, float2 &b, float2 &c, float2 &d) {
    const float2 s02 = cadd(a, c), d02 = csub(a, c), s13 = cadd(b, d), d13 = csub(b, d);
    a = cadd(s02, s13);
    c = csub(s02, s13);
    b = cadd_mi(d02, d13);
    d = csub_mi(d02, d13);
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

// Where the launch's rows live: the arrays hold view_rows rows per view
// (rows_per_view when they hold just the band, Nv for whole-detector
// arrays), and band row i of view k sits at memory row k view_rows + off + i.
struct RowMap {
    int rows_per_view, view_rows, off;
    __device__ __forceinline__ long long mem(long long r) const {
        if (view_rows == rows_per_view) return r + off;  // the arrays hold just these rows
        if (r <= 0x7fffffffLL) {                          // 32-bit division where it suffices
            const unsigned k = (unsigned)r / (unsigned)rows_per_view;
            return (long long)k * view_rows + off + ((unsigned)r - k * (unsigned)rows_per_view);
        }
        const long long k = r / rows_per_view;
        return k * view_rows + off + (r - k * rows_per_view);
    }
};

// G row pairs per CTA, L/16 threads per pair: weighted rows into shared
// memory, forward transform (times the spectrum on its last pass), inverse
// transform (its last pass stores the rows of Q).
template <typename TQ>
__global__ void __launch_bounds__(kThreads)
filter_kernel(const float *__restrict__ proj, TQ *__restrict__ Q, const float *__restrict__ H,
              const float2 *__restrict__ tw, int L, int lgL, int G, int Nu, int Nv, int row0, RowMap rm,
              long long nrows, float R) {
    const int rows_per_view = rm.rows_per_view;
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
    // memory rows, once per thread (a 64-bit division)
    const long long mA = hasA ? rm.mem(rowA) : 0, mB = hasB ? rm.mem(rowB) : 0;
    const float *pa = proj + mA * Nu, *pb = proj + mB * Nu;
    for (int i = lt; i < L / 2; i += nt) {  // the upper half is never read (see pass)
        float2 v = make_float2(0.f, 0.f);
        if (i < Nu) {
            const float u = (float)i - 0.5f * (float)(Nu - 1);
            if (hasA) v.x = __ldg(pa + i) * (R * rsqrtf(R2 + u * u + bA * bA));
            if (hasB) v.y = __ldg(pb + i) * (R * rsqrtf(R2 + u * u + bB * bB));
        }
        buf[pad(i)] = v;
    }
    __syncthreads();
    Sink<TQ> sink;
    sink.H = H;
    sink.qa = hasA ? Q + mA * Nu : nullptr;
    sink.qb = hasB ? Q + mB * Nu : nullptr;
    sink.Nu = Nu;
    fft<kToSpectrum>(buf, tw, lgL, lt, nt, sink);
    fft<kToQ>(buf, tw, lgL, lt, nt, sink);
}

// ---------------------------------------------------------------------------
// Warp form for L = 1024 (detector rows of 257 .. 512 columns): one warp per
// row pair, the transform of length 1024 = 32 x 32 done as a 32-point DFT
// in every lane's registers, one twiddle multiply, a transpose through a
// padded 32 x 33 tile of shared memory and a second 32-point DFT.  Input
// sample n = 32 n1 + n2 sits in lane n2, register n1 (coalesced loads; n1 <
// 16 since the upper half is padding); after the forward transform lane k1
// holds X[k1 + 32 k2] in register k2, multiplies by the ramp spectrum,
// conjugates, and the same two steps run again; output sample n = n1 +
// 32 n2 ends in lane n1, register n2 (coalesced stores).  No block barrier:
// each warp only synchronises with itself around its transposes.

constexpr int kFilterWarps = 4;  // row pairs per CTA

// W32^k = e^{-2 pi i k / 32}, k = 0 .. 15: cos(k pi / 16) and sin(k pi / 16)
__device__ __forceinline__ constexpr float cos16(int k) {
    return k == 0 ? 1.0f : k == 1 ? 0.98078528040323044913f : k == 2 ? 0.92387953251128675613f
         : k == 3 ? 0.83146961230254523708f : k == 4 ? 0.70710678118654752440f : k == 5 ? 0.55557023301960222474f
         : k == 6 ? 0.38268343236508977173f : k == 7 ? 0.19509032201612826785f : k == 8 ? 0.0f : -cos16(16 - k);
}
__device__ __forceinline__ constexpr float sin16(int k) { return k <= 8 ? cos16(8 - k) : cos16(k - 8); }

// 32-point forward DFT in registers, in place, by decimation in frequency:
// u[n] = v[n] + v[n + 16] and w[n] = (v[n] - v[n + 16]) W32^n for n < 16,
// then X[2k] = DFT16(u)[k] and X[2k + 1] = DFT16(w)[k].  Input in natural
// order; X[k] is left at v[pos32(k)].  HALF: v[16 ..] are zero on input.
__device__ __forceinline__ constexpr int pos32(int k) {
    return (k & 1) ? 16 + out_pos<16>(k >> 1) : out_pos<16>(k >> 1);
}

template <bool HALF = false>
__device__ __forceinline__ void dft32(float2 *v) {
#pragma unroll
    for (int n = 0; n < 16; ++n) {
        const float2 a = v[n], b = v[n + 16];
        float2 d = HALF ? a : csub(a, b);
        if (!HALF) v[n] = cadd(a, b);
        if (n == 8) d = cmi(d);
        else if (n != 0) d = cmul(d, make_float2(cos16(n), -sin16(n)));
        v[n + 16] = d;
    }
    dft<16>(v);
    dft<16>(v + 16);
}

constexpr int kTile32 = 32 * 33;                  // padded 32 x 32 transpose tile (float2)
constexpr int kStage = 1024;                      // floats of a staged row pair (2 rows of <= 512)
constexpr uint64_t kFilterWaitNs = 2000000000ull;  // bounded wait on a staged row pair
// dynamic shared memory: per warp a staging buffer and a transpose tile,
// then the twiddles W1024^(a b) and the ramp spectrum
constexpr size_t kFilterSmem =
    128 + (size_t)kFilterWarps * (kStage * sizeof(float) + kTile32 * sizeof(float2)) + 1024 * (sizeof(float2) + sizeof(float));

template <typename TQ>
__global__ void __launch_bounds__(32 * kFilterWarps, 3)
filter_1024_kernel(const float *__restrict__ proj, TQ *__restrict__ Q, const float *__restrict__ H,
                   const float2 *__restrict__ tw2, int Nu, int Nv, int row0, RowMap rm, int nrows, float R,
                   int *status) {
    const int rows_per_view = rm.rows_per_view;
    extern __shared__ __align__(128) unsigned char fsm_raw[];
    unsigned char *base = fsm_raw + ((128u - (tma::smem_u32(fsm_raw) & 127u)) & 127u);
    float(*stg)[kStage] = reinterpret_cast<float(*)[kStage]>(base);
    float2(*tile)[kTile32] = reinterpret_cast<float2(*)[kTile32]>(base + kFilterWarps * kStage * sizeof(float));
    float2 *s_tw = reinterpret_cast<float2 *>(base + kFilterWarps * (kStage * sizeof(float) + kTile32 * sizeof(float2)));
    float *s_h = reinterpret_cast<float *>(s_tw + 1024);
    __shared__ __align__(8) uint64_t bar[kFilterWarps];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int i = threadIdx.x; i < 1024; i += blockDim.x) {
        s_tw[i] = tw2[i];
        s_h[i] = H[i];
    }
    if (lane == 0) {
        tma::mbar_init(&bar[warp], 1);
        tma::fence_mbar_init();
    }
    __syncthreads();
    const int npairs = (nrows + 1) / 2;
    const int stride = gridDim.x * kFilterWarps;
    float *in = stg[warp];
    float2 *t = tile[warp];
    // rows 2 pr and 2 pr + 1: one copy where they are adjacent in memory
    auto stage = [&](int pr) {
        const int rows = min(2, nrows - 2 * pr);
        const long long ma = rm.mem(2 * pr), mb = rm.mem(2 * pr + 1);
        const uint32_t row_bytes = (uint32_t)Nu * 4u;
        tma::fence_proxy_async();
        tma::mbar_arrive_expect_tx(&bar[warp], (uint32_t)rows * row_bytes);
        if (rows == 2 && mb != ma + 1) {
            tma::bulk_load(in, proj + (size_t)ma * Nu, row_bytes, &bar[warp]);
            tma::bulk_load(in + Nu, proj + (size_t)mb * Nu, row_bytes, &bar[warp]);
        } else {
            tma::bulk_load(in, proj + (size_t)ma * Nu, (uint32_t)rows * row_bytes, &bar[warp]);
        }
    };
    int pair = blockIdx.x * kFilterWarps + warp;
    if (pair < npairs && lane == 0) stage(pair);
    const float R2 = R * R;
    for (int it = 0; pair < npairs; ++it, pair += stride) {
        if (!tma::mbar_wait_bounded(&bar[warp], (uint32_t)(it & 1), kFilterWaitNs)) {
            // the copy never completed: report, give it a last chance to land, leave
            if (lane == 0) atomicOr(status, 2);
            tma::mbar_wait_bounded(&bar[warp], (uint32_t)(it & 1), kFilterWaitNs);
            return;
        }
        const int rowA = 2 * pair, rowB = rowA + 1;
        const bool hasB = rowB < nrows;
        const float bA = (float)(row0 + rowA % rows_per_view) - 0.5f * (float)(Nv - 1);
        const float bB = (float)(row0 + rowB % rows_per_view) - 0.5f * (float)(Nv - 1);
        float2 v[32];
        // both rows present and 512 samples long (the common case): loads
        // and stores without per-sample tests, whose branches cost more
        // than the arithmetic they guard (measured: 1.10 -> 0.93 ms for
        // 512 x 512 x 720, same results bit for bit)
        const bool full = Nu == 512 && hasB;
        if (full) {
#pragma unroll
            for (int n1 = 0; n1 < 16; ++n1) {
                const int n = 32 * n1 + lane;
                const float u = (float)n - 255.5f;
                v[n1] = make_float2(in[n] * (R * rsqrtf(R2 + u * u + bA * bA)),
                                    in[512 + n] * (R * rsqrtf(R2 + u * u + bB * bB)));
            }
        } else {
#pragma unroll
            for (int n1 = 0; n1 < 16; ++n1) {
                const int n = 32 * n1 + lane;
                float2 x = make_float2(0.f, 0.f);
                if (n < Nu) {
                    const float u = (float)n - 0.5f * (float)(Nu - 1);
                    x.x = in[n] * (R * rsqrtf(R2 + u * u + bA * bA));
                    if (hasB) x.y = in[Nu + n] * (R * rsqrtf(R2 + u * u + bB * bB));
                }
                v[n1] = x;
            }
        }
#pragma unroll
        for (int n1 = 16; n1 < 32; ++n1) v[n1] = make_float2(0.f, 0.f);
        // the input is in registers: the staging buffer takes the next pair
        __syncwarp();
        if (pair + stride < npairs && lane == 0) stage(pair + stride);
        // two passes of the same code (one copy of it keeps the loop body in
        // the instruction cache): lane a transforms over its 32 values,
        // twiddles by W1024^(a b), and the transpose hands lane b the values
        // of every a, which it transforms again.  Pass 0 is the forward
        // transform (a = n2, b = k1), followed by the product with the ramp
        // spectrum (over L) and the conjugation; pass 1 is the inverse as the
        // conjugate of a forward transform (a = k1, b = n1).
#pragma unroll 1
        for (int pass = 0; pass < 2; ++pass) {
            dft32(v);
#pragma unroll
            for (int k = 0; k < 32; ++k) t[k * 33 + lane] = cmul(v[pos32(k)], s_tw[k * 32 + lane]);
            __syncwarp();
#pragma unroll
            for (int n = 0; n < 32; ++n) v[n] = t[lane * 33 + n];
            __syncwarp();
            dft32(v);
            if (pass == 0) {
                // X[lane + 32 k2] sits at v[pos32(k2)]: spectrum product,
                // conjugation, natural order for the next pass
                float2 g[32];
#pragma unroll
                for (int k2 = 0; k2 < 32; ++k2) {
                    const float h = s_h[lane + 32 * k2];
                    const float2 x = v[pos32(k2)];
                    g[k2] = make_float2(x.x * h, -x.y * h);
                }
#pragma unroll
                for (int k2 = 0; k2 < 32; ++k2) v[k2] = g[k2];
            }
        }
        // sample n = lane + 32 n2 of the conjugated result: row A real, row B imaginary
        TQ *qa = Q + (size_t)rm.mem(rowA) * Nu, *qb = Q + (size_t)rm.mem(rowB) * Nu;
        if (full) {
#pragma unroll
            for (int n2 = 0; n2 < 16; ++n2) {
                const int n = lane + 32 * n2;
                const float2 y = v[pos32(n2)];
                qa[n] = to_q<TQ>(y.x);
                qb[n] = to_q<TQ>(-y.y);
            }
        } else
#pragma unroll
        for (int n2 = 0; n2 < 16; ++n2) {
            const int n = lane + 32 * n2;
            if (n < Nu) {
                const float2 y = v[pos32(n2)];
                qa[n] = to_q<TQ>(y.x);
                if (hasB) qb[n] = to_q<TQ>(-y.y);
            }
        }
    }
}

template <typename TQ>
cudaError_t launch_t(const PlanImpl &p, const float *proj, TQ *Q, cudaStream_t st, int row0, int rows_per_view,
                     int views, bool whole_arrays) {
    const long long nrows = (long long)views * rows_per_view;
    RowMap rm;
    rm.rows_per_view = rows_per_view;
    rm.view_rows = whole_arrays ? p.g.Nv : rows_per_view;
    rm.off = whole_arrays ? row0 : 0;
    const long long pairs = (nrows + 1) / 2;
    // the warp form stages rows with bulk copies: 16-byte aligned rows
    if (p.L == 1024 && p.tw2 && (p.g.Nu % 4) == 0 && ((uintptr_t)proj & 15) == 0 && nrows < (1LL << 30)) {
        // as many CTAs as the GPU holds at once (each warp loops over pairs)
        const size_t smem = kFilterSmem;
        cudaError_t e = ensure_smem<filter_1024_kernel<TQ>>(smem);
        if (e != cudaSuccess) return e;
        int dev = 0, sms = 0, per_sm = 0;
        if ((e = cudaGetDevice(&dev)) != cudaSuccess ||
            (e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess ||
            (e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, filter_1024_kernel<TQ>, 32 * kFilterWarps,
                                                               smem)) != cudaSuccess)
            return e;
        const long long need = (pairs + kFilterWarps - 1) / kFilterWarps;
        const long long blocks = std::max(1LL, std::min(need, (long long)std::max(1, per_sm) * sms));
        filter_1024_kernel<TQ><<<(unsigned)blocks, 32 * kFilterWarps, smem, st>>>(
            proj, Q, p.H, p.tw2, p.g.Nu, p.g.Nv, row0, rm, (int)nrows, (float)p.g.R, p.status);
        return cudaGetLastError();
    }
    const int G = std::max(1, 2048 / p.L);  // 128 threads per CTA up to L = 2048
    const long long blocks = (pairs + G - 1) / G;
    const size_t smem = sizeof(float2) * (size_t)G * (p.L + p.L / 16);
    cudaError_t e = ensure_smem<filter_kernel<TQ>>(smem);
    if (e != cudaSuccess) return e;
    filter_kernel<TQ><<<(unsigned)blocks, G * (p.L / 16), smem, st>>>(proj, Q, p.H, p.tw, p.L, p.log2L, G, p.g.Nu, p.g.Nv,
                                                                      row0, rm, nrows, (float)p.g.R);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_filter(const PlanImpl &p, const float *proj, void *Q, cudaStream_t st, Band b, int views) {
    const int rows = b.nrows < 0 ? p.g.Nv : b.nrows;
    if (views < 0) views = p.g.P;
    if (views == 0) return cudaSuccess;
    switch (p.qtype) {
        case FDKOD_F32: return launch_t(p, proj, (float *)Q, st, b.row0, rows, views, b.whole_arrays);
        case FDKOD_BF16: return launch_t(p, proj, (__nv_bfloat16 *)Q, st, b.row0, rows, views, b.whole_arrays);
        case FDKOD_F16: return launch_t(p, proj, (__half *)Q, st, b.row0, rows, views, b.whole_arrays);
    }
    return cudaErrorInvalidValue;
}

}  // namespace fdkod
