// Per-(square, view) crop bounds: Eq. 1 evaluated at the four vertices of
// each of the 4^s squares (Sec. 2.1, Sec. 2.2), in FP64 with explicit
// round-to-nearest operations (no contraction) so that the integer bounds
// are reproducible bit for bit against any FP64 evaluation of Eq. 1 in the
// same operation order.  Trigonometry comes from host tables.
#include <math.h>

#include "fdkod_internal.cuh"

namespace fdkod {
namespace {

// Eq. 1, evaluated left to right as printed:
// a = R (y cos b - x sin b) / (R + x cos b + y sin b).
__device__ __forceinline__ double eq1(double R, double x, double y, double cb, double sb) {
    double num = __dsub_rn(__dmul_rn(y, cb), __dmul_rn(x, sb));
    double den = __dadd_rn(__dadd_rn(R, __dmul_rn(x, cb)), __dmul_rn(y, sb));
    return __ddiv_rn(__dmul_rn(R, num), den);
}

__device__ __forceinline__ double vcentre(int i, int n) {
    return __dsub_rn((double)i, __dmul_rn(0.5, (double)(n - 1)));
}

__device__ __forceinline__ void square_range(int q, int m, int N, int &i0, int &i1) {
    i0 = (int)(((long long)q * N + m - 1) / m);
    i1 = (int)((((long long)q + 1) * N + m - 1) / m) - 1;
}

constexpr int kThreads = 256;

// One CTA per square; threads stride over the views.
__global__ void __launch_bounds__(kThreads)
bounds_kernel(double R, int N, int Nu, int P, int m, const double2 *__restrict__ cs,
              int32_t *__restrict__ lo, int32_t *__restrict__ hi, int32_t *__restrict__ crop,
              double *__restrict__ phi, int32_t *__restrict__ w0o, int32_t *__restrict__ To,
              GeomEntry *__restrict__ geo) {
    const int q = blockIdx.x;
    const int qy = q / m, qx = q % m;
    int ix0, ix1, iy0, iy1;
    square_range(qx, m, N, ix0, ix1);
    square_range(qy, m, N, iy0, iy1);
    const double xs[2] = {vcentre(ix0, N), vcentre(ix1, N)};
    const double ys[2] = {vcentre(iy0, N), vcentre(iy1, N)};
    const double xc = __dmul_rn(0.5, __dadd_rn(xs[0], xs[1]));
    const double yc = __dmul_rn(0.5, __dadd_rn(ys[0], ys[1]));
    const double uc = __dmul_rn(0.5, (double)(Nu - 1));

    double dmin = INFINITY, dmax = -INFINITY;
    for (int k = threadIdx.x; k < P; k += kThreads) {
        const double cb = cs[k].x, sb = cs[k].y;
        double umin = INFINITY, umax = -INFINITY;
#pragma unroll
        for (int vy = 0; vy < 2; ++vy)
#pragma unroll
            for (int vx = 0; vx < 2; ++vx) {
                double u = __dadd_rn(eq1(R, xs[vx], ys[vy], cb, sb), uc);
                umin = fmin(umin, u);
                umax = fmax(umax, u);
            }
        const double p = __dadd_rn(eq1(R, xc, yc, cb, sb), uc);
        const size_t o = (size_t)q * P + k;
        lo[o] = (int32_t)floor(umin);
        hi[o] = (int32_t)floor(umax) + 1;
        phi[o] = p;
        dmin = fmin(dmin, __dsub_rn(umin, p));
        dmax = fmax(dmax, __dsub_rn(umax, p));
    }
    // min / max are exact, so the reduction order does not matter
    __shared__ double smin[kThreads / 32], smax[kThreads / 32];
    __shared__ int32_t sw0;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        dmin = fmin(dmin, __shfl_xor_sync(0xffffffffu, dmin, off));
        dmax = fmax(dmax, __shfl_xor_sync(0xffffffffu, dmax, off));
    }
    if ((threadIdx.x & 31) == 0) {
        smin[threadIdx.x >> 5] = dmin;
        smax[threadIdx.x >> 5] = dmax;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = smin[0], b = smax[0];
        for (int i = 1; i < kThreads / 32; ++i) {
            a = fmin(a, smin[i]);
            b = fmax(b, smax[i]);
        }
        const int32_t w = (int32_t)floor(a) - 1;
        sw0 = w;
        w0o[q] = w;
        To[q] = (int32_t)floor(b) + 3 - w;
    }
    __syncthreads();
    const int32_t w = sw0;
    for (int k = threadIdx.x; k < P; k += kThreads) {
        const double cb = cs[k].x, sb = cs[k].y;
        const double p = __dadd_rn(eq1(R, xc, yc, cb, sb), uc);
        const double pw = __dadd_rn(p, (double)w);
        const double c = floor(pw);
        const size_t o = (size_t)q * P + k;
        crop[o] = (int32_t)c;
        // FP32 backprojection coefficients (not part of the bit-exact set)
        const double dc = R + xc * cb + yc * sb;
        const double e = (yc * cb - xc * sb) / dc;
        GeomEntry ge;
        const double g = R / dc;
        ge.g_hi = (float)g;
        ge.g_lo = (float)(g - (double)ge.g_hi);
        ge.cb = (float)cb;
        ge.sb = (float)sb;
        ge.r = (float)(1.0 / dc);
        ge.alpha = (float)(-sb - e * cb);
        ge.gamma = (float)(cb - e * sb);
        ge.frac = (float)(pw - c);
        geo[o] = ge;
    }
}

}  // namespace

cudaError_t launch_bounds(const PlanImpl &p, SquareSet &ss, cudaStream_t st) {
    bounds_kernel<<<ss.nsq, kThreads, 0, st>>>(p.g.R, p.g.N, p.g.Nu, p.g.P, ss.m, p.cs, ss.lo, ss.hi,
                                               ss.crop, ss.phi, ss.w0, ss.T, ss.geo);
    return cudaGetLastError();
}

}  // namespace fdkod
