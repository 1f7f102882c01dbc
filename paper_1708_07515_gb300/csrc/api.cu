// C ABI of libfdkod: plan construction (host-side validation, trig tables,
// FFT tables, workspace sizing) and the entry points of include/fdkod.h.
#include <math.h>
#include <cmath>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "fdkod_internal.cuh"
#include "tma.cuh"

using namespace fdkod;

#include <cudaTypedefs.h>

namespace {

int cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return FDKOD_OK;
    return e == cudaErrorMemoryAllocation ? FDKOD_ERR_OOM : FDKOD_ERR_CUDA;
}

#define FDKOD_TRY(expr)                           \
    do {                                          \
        int _rc = cuda_status(expr);              \
        if (_rc != FDKOD_OK) return _rc;          \
    } while (0)

template <typename T>
cudaError_t dalloc(PlanImpl &p, T **ptr, size_t n) {
    cudaError_t e = cudaMalloc((void **)ptr, sizeof(T) * std::max<size_t>(n, 1));
    if (e == cudaSuccess) p.device_bytes += (int64_t)(sizeof(T) * std::max<size_t>(n, 1));
    return e;
}

void free_set(SquareSet &ss) {
    cudaFree(ss.lo);
    cudaFree(ss.hi);
    cudaFree(ss.crop);
    cudaFree(ss.w0);
    cudaFree(ss.T);
    cudaFree(ss.phi);
    cudaFree(ss.geo);
    ss = SquareSet{};
}

void free_plan(PlanImpl &p) {
    free_set(p.od);
    free_set(p.pl);
    cudaFree(p.cs);
    cudaFree(p.H);
    cudaFree(p.tw);
    cudaFree(p.tw2);
    cudaFree(p.Sp);
    cudaFree(p.tapw);
    cudaFree(p.net);
    cudaFree(p.status);
    free_host_pipe(p.pipe);
    p.pipe = nullptr;
    free_slab_pipe(p.slabs);
    p.slabs = nullptr;
}

double centre(int i, int n) { return (double)i - 0.5 * (double)(n - 1); }

void square_range(int q, int m, int N, int &i0, int &i1) {
    i0 = (int)(((long long)q * N + m - 1) / m);
    i1 = (int)((((long long)q + 1) * N + m - 1) / m) - 1;
}

}  // namespace

namespace fdkod {

// Staging window of the backprojection kernel: the largest column and row
// extent any 16 x 16 x kZT voxel tile of this square set can touch in one
// view, from an FP64 sweep over all tiles and views (column coordinate
// relative to the square centre; row extent bounded over all slabs).
void size_windows(const PlanImpl &p, SquareSet &ss, const double2 *cs) {
    const double R = p.g.R;
    const int N = p.g.N, P = p.g.P;
    const int mside = (N + ss.m - 1) / ss.m;
    ss.tiles_per_side = (mside + kTile - 1) / kTile;
    double ext_t = 0.0, ext_v = 0.0, ext_v2 = 0.0;
    // the last slab's tile may run kZT slices past the volume
    const double zabs = 0.5 * (double)(N - 1) + kZT;
    for (int q = 0; q < ss.nsq; ++q) {
        int ix0, ix1, iy0, iy1;
        square_range(q % ss.m, ss.m, N, ix0, ix1);
        square_range(q / ss.m, ss.m, N, iy0, iy1);
        const double xc = 0.5 * (centre(ix0, N) + centre(ix1, N));
        const double yc = 0.5 * (centre(iy0, N) + centre(iy1, N));
        for (int ty = iy0; ty <= iy1; ty += kTile)
            for (int tx = ix0; tx <= ix1; tx += kTile) {
                const double xs[2] = {centre(tx, N), centre(std::min(tx + kTile - 1, ix1), N)};
                const double ys[2] = {centre(ty, N), centre(std::min(ty + kTile - 1, iy1), N)};
                for (int k = 0; k < P; ++k) {
                    const double cb = cs[k].x, sb = cs[k].y;
                    const double ac = R * (yc * cb - xc * sb) / (R + xc * cb + yc * sb);
                    double tmin = 1e300, tmax = -1e300, umin = 1e300, umax = -1e300;
                    for (int a = 0; a < 2; ++a)
                        for (int b = 0; b < 2; ++b) {
                            const double den = R + xs[a] * cb + ys[b] * sb;
                            const double t = R * (ys[b] * cb - xs[a] * sb) / den - ac;
                            const double iu = R / den;
                            tmin = std::min(tmin, t);
                            tmax = std::max(tmax, t);
                            umin = std::min(umin, iu);
                            umax = std::max(umax, iu);
                        }
                    ext_t = std::max(ext_t, tmax - tmin);
                    ext_v = std::max(ext_v, (double)(kZT - 1) * umax + zabs * (umax - umin));
                    ext_v2 = std::max(ext_v2, (double)(kZP - 1) * umax + zabs * (umax - umin));
                }
            }
    }
    // floor(max) - floor(min) <= ceil(extent); +2 for the interpolation
    // neighbour and the one-sample margin below; +2 for FP32 rounding slack
    ss.Wd = (int)ceil(ext_t) + 5;
    ss.Wd += ss.Wd & 1;  // even width: odd shared-memory row stride
    ss.Rw = (int)ceil(ext_v) + 5;
    ss.Rw2 = (int)ceil(ext_v2) + 5;
    // TMA copies start on a 16-byte boundary: up to 3 more float32 columns,
    // or 7 more 16-bit columns
    const int need = (int)ceil(ext_t) + 8, need16 = (int)ceil(ext_t) + 12;
    ss.need = need;
    ss.need16 = need16;
    ss.WdT = ss.WdT16 = 0;
    for (int w : {128, 96, 64, 48, 32}) {
        if (need <= w) ss.WdT = w;
        if (need16 <= w) ss.WdT16 = w;
    }
}

void triangle_taps(int D, double *h) {
    for (int i = 0; i < D; ++i) h[i] = (double)(D - i) / ((double)D * (double)D);
}

void sinc_taps(int D, int H, double *h) {
    // g_i = sinc(i / D) (1 + cos(pi i / (H D))) / 2, |i| < H D, scaled so the
    // two-sided sum (the response at zero frequency) is 1
    const int n = H * D;
    double sum = 0.0;
    for (int i = 0; i < n; ++i) {
        const double x = (double)i / (double)D;
        const double sinc = i == 0 ? 1.0 : sin(M_PI * x) / (M_PI * x);
        h[i] = sinc * 0.5 * (1.0 + cos(M_PI * (double)i / (double)n));
        sum += i == 0 ? h[i] : 2.0 * h[i];
    }
    for (int i = 0; i < n; ++i) h[i] /= sum;
}

void tap_table(const double *h, int H, int D, float4 *w) {
    for (int r = 0; r < D; ++r) {
        float v[4] = {0.f, 0.f, 0.f, 0.f};
        for (int m = 0; m < 2 * H; ++m) {
            const int o = std::abs(r + (H - 1 - m) * D);
            v[m] = o < H * D ? (float)h[o] : 0.f;
        }
        w[r] = make_float4(v[0], v[1], v[2], v[3]);
    }
}

}  // namespace fdkod

namespace {

int make_set(PlanImpl &p, SquareSet &ss, int s, cudaStream_t st, const std::vector<double2> &cs) {
    ss.s = s;
    ss.m = 1 << s;
    ss.nsq = ss.m * ss.m;
    const size_t n = (size_t)ss.nsq * p.g.P;
    FDKOD_TRY(dalloc(p, &ss.lo, n));
    FDKOD_TRY(dalloc(p, &ss.hi, n));
    FDKOD_TRY(dalloc(p, &ss.crop, n));
    FDKOD_TRY(dalloc(p, &ss.phi, n));
    FDKOD_TRY(dalloc(p, &ss.geo, n));
    FDKOD_TRY(dalloc(p, &ss.w0, (size_t)ss.nsq));
    FDKOD_TRY(dalloc(p, &ss.T, (size_t)ss.nsq));
    FDKOD_TRY(launch_bounds(p, ss, st));
    std::vector<int32_t> T(ss.nsq);
    FDKOD_TRY(cudaMemcpyAsync(T.data(), ss.T, sizeof(int32_t) * ss.nsq, cudaMemcpyDeviceToHost, st));
    FDKOD_TRY(cudaStreamSynchronize(st));
    ss.Tmax = *std::max_element(T.begin(), T.end());
    size_windows(p, ss, cs.data());
    return FDKOD_OK;
}

// Discrete Ram-Lak kernel, unit sample spacing.
double ramlak(long n) {
    if (n == 0) return 0.25;
    if (n % 2 == 0) return 0.0;
    return -1.0 / (M_PI * M_PI * (double)n * (double)n);
}

int make_fft_tables(PlanImpl &p, cudaStream_t st) {
    int L = 1, lg = 0;
    while (L < 2 * p.g.Nu) {
        L <<= 1;
        ++lg;
    }
    if (L < 16) {  // the filter's transforms start with a radix-16 pass
        L = 16;
        lg = 4;
    }
    p.L = L;
    p.log2L = lg;
    // kernel wrapped onto the circle of length L (taps |n| <= L/2); as
    // L >= 2 Nu every product of the linear convolution sits at its own lag
    std::vector<double> ctab(L);
    for (int i = 0; i < L; ++i) ctab[i] = cos(2.0 * M_PI * (double)i / (double)L);
    std::vector<float> H(L);
    for (int k = 0; k < L; ++k) {
        double acc = ramlak(0);
        for (int n = 1; n < L / 2; n += 2) acc += 2.0 * ramlak(n) * ctab[(size_t)((long long)k * n % L)];
        acc += ramlak(L / 2) * ctab[(size_t)((long long)k * (L / 2) % L)];
        H[k] = (float)(acc / (double)L);
    }
    std::vector<float2> tw(L);
    for (int i = 0; i < L; ++i) {
        const double a = 2.0 * M_PI * (double)i / (double)L;
        tw[i] = make_float2((float)cos(a), (float)(-sin(a)));
    }
    FDKOD_TRY(dalloc(p, &p.H, (size_t)L));
    FDKOD_TRY(dalloc(p, &p.tw, (size_t)L));
    FDKOD_TRY(cudaMemcpyAsync(p.H, H.data(), sizeof(float) * L, cudaMemcpyHostToDevice, st));
    FDKOD_TRY(cudaMemcpyAsync(p.tw, tw.data(), sizeof(float2) * L, cudaMemcpyHostToDevice, st));
    std::vector<float2> tw2;
    if (L == 1024) {  // the warp transform's twiddles W^(a b), a, b < 32
        tw2.resize(1024);
        for (int a = 0; a < 32; ++a)
            for (int b = 0; b < 32; ++b) {
                const double ang = 2.0 * M_PI * (double)(a * b) / 1024.0;
                tw2[(size_t)a * 32 + b] = make_float2((float)cos(ang), (float)(-sin(ang)));
            }
        FDKOD_TRY(dalloc(p, &p.tw2, tw2.size()));
        FDKOD_TRY(cudaMemcpyAsync(p.tw2, tw2.data(), sizeof(float2) * tw2.size(), cudaMemcpyHostToDevice, st));
    }
    FDKOD_TRY(cudaStreamSynchronize(st));
    return FDKOD_OK;
}

int build_plan(PlanImpl &p, cudaStream_t st) {
    const int P = p.g.P;
    std::vector<double2> cs(P);
    for (int k = 0; k < P; ++k) {
        const double beta = 2.0 * M_PI * (double)k / (double)P;
        cs[k] = make_double2(cos(beta), sin(beta));
    }
    FDKOD_TRY(dalloc(p, &p.cs, (size_t)P));
    FDKOD_TRY(cudaMemcpyAsync(p.cs, cs.data(), sizeof(double2) * P, cudaMemcpyHostToDevice, st));
    FDKOD_TRY(dalloc(p, &p.status, 1));
    FDKOD_TRY(cudaMemsetAsync(p.status, 0, sizeof(int), st));
    int rc = make_set(p, p.od, p.s, st, cs);
    if (rc) return rc;
    // plain FDK tiling: squares of 64..127 voxels a side (whole slice when
    // N < 128), cut into 16 x 16 tiles
    int sp = 0;
    while ((p.g.N >> (sp + 1)) >= 64 && sp < 7) ++sp;
    rc = make_set(p, p.pl, sp, st, cs);
    if (rc) return rc;
    rc = make_fft_tables(p, st);
    if (rc) return rc;
    p.Tstride = (p.od.Tmax + 3) & ~3;
    // angular low-pass of the decomposition
    if (p.tap_blocks == 2) sinc_taps(p.D, 2, p.htaps);
    else triangle_taps(p.D, p.htaps);
    {
        std::vector<float4> w(p.D);
        tap_table(p.htaps, p.tap_blocks, p.D, w.data());
        FDKOD_TRY(dalloc(p, &p.tapw, (size_t)p.D));
        FDKOD_TRY(cudaMemcpyAsync(p.tapw, w.data(), sizeof(float4) * p.D, cudaMemcpyHostToDevice, st));
        FDKOD_TRY(cudaStreamSynchronize(st));
    }
    if (p.D > 1 && !p.no_workspace) {
        p.sp_elems = (int64_t)p.od.nsq * p.Pd * p.g.Nv * p.Tstride;
        FDKOD_TRY(dalloc(p, &p.Sp, (size_t)p.sp_elems));
    }
    FDKOD_TRY(cudaStreamSynchronize(st));
    return FDKOD_OK;
}

PFN_cuTensorMapEncodeTiled_v12000 get_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *ptr = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)ptr;
    }
    return fn;
}

bool valid_dtype(int t) { return t == FDKOD_F32 || t == FDKOD_BF16 || t == FDKOD_F16; }

}  // namespace

namespace fdkod {

cudaError_t encode_map_3d(CUtensorMap *map, CUtensorMapDataType dt, const void *base, const uint64_t dims[3],
                          const uint64_t strides[2], const uint32_t box[3]) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = get_encoder();
    if (!enc) return cudaErrorNotSupported;
    const cuuint64_t gd[3] = {dims[0], dims[1], dims[2]};
    const cuuint64_t gs[2] = {strides[0], strides[1]};
    const cuuint32_t bx[3] = {box[0], box[1], box[2]};
    const cuuint32_t es[3] = {1, 1, 1};
    CUresult r = enc(map, dt, 3, const_cast<void *>(base), gd, gs, bx, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

}  // namespace fdkod

extern "C" {

int fdkod_plan(const fdkod_geometry *g, int s, int D, fdkod_dtype qtype, fdkod_plan_t **out) {
    return fdkod_plan_ex(g, s, D, qtype, 0, out);
}

int fdkod_plan_ex(const fdkod_geometry *g, int s, int D, fdkod_dtype qtype, int flags, fdkod_plan_t **out) {
    if (!g || !out) return FDKOD_ERR_INVALID_ARG;
    *out = nullptr;
    if (flags & ~(FDKOD_PLAN_NO_WORKSPACE | FDKOD_PLAN_SINC_TAPS)) return FDKOD_ERR_INVALID_ARG;
    if (!(g->R > 0.0) || g->N <= 0 || g->Nu <= 0 || g->Nv <= 0 || g->P <= 0 || D <= 0 || !valid_dtype(qtype))
        return FDKOD_ERR_INVALID_ARG;
    const int lim = 1 << 15;
    if (g->N > lim || g->Nu > lim || g->Nv > lim || g->P > lim) return FDKOD_ERR_UNSUPPORTED;
    // the filter's shared-memory FFT of length L = 2^ceil(log2(2 Nu)) uses
    // one thread per 16 samples (at most 1024: L <= 16384) and L (1 + 1/16)
    // complex floats of shared memory (139 KiB at L = 16384)
    if (g->Nu > 8192) return FDKOD_ERR_UNSUPPORTED;
    if (s < 0 || s > 7 || (1 << s) > g->N || g->P % D != 0 || D > fdkod::kMaxTapD) return FDKOD_ERR_UNSUPPORTED;
    // the source must lie outside the volume's circumscribed cylinder
    if (!(g->R > M_SQRT2 * 0.5 * (double)g->N + 1.0)) return FDKOD_ERR_UNSUPPORTED;
    fdkod_plan_t *pl = new (std::nothrow) fdkod_plan_t;
    if (!pl) return FDKOD_ERR_OOM;
    PlanImpl &p = pl->impl;
    p.g = *g;
    p.s = s;
    p.D = D;
    p.Pd = g->P / D;
    p.qtype = qtype;
    p.no_workspace = (flags & FDKOD_PLAN_NO_WORKSPACE) != 0;
    p.tap_blocks = (flags & FDKOD_PLAN_SINC_TAPS) && D > 1 ? 2 : 1;
    cudaStream_t st;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
        delete pl;
        return FDKOD_ERR_CUDA;
    }
    int rc = build_plan(p, st);
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
    if (rc != FDKOD_OK) {
        free_plan(p);
        delete pl;
        return rc;
    }
    *out = pl;
    return FDKOD_OK;
}

void fdkod_destroy(fdkod_plan_t *plan) {
    if (!plan) return;
    cudaDeviceSynchronize();
    free_plan(plan->impl);
    delete plan;
}

int fdkod_get_info(const fdkod_plan_t *plan, fdkod_plan_info *info) {
    if (!plan || !info) return FDKOD_ERR_INVALID_ARG;
    const PlanImpl &p = plan->impl;
    info->s = p.s;
    info->D = p.D;
    info->Pd = p.Pd;
    info->n_squares = p.od.nsq;
    info->T_stride = p.Tstride;
    info->fft_length = p.L;
    info->decomposed_elems = (int64_t)p.od.nsq * p.Pd * p.g.Nv * p.Tstride * (p.D > 1 ? 1 : 0);
    info->device_bytes = p.device_bytes;
    return FDKOD_OK;
}

int fdkod_filter(fdkod_plan_t *plan, const float *proj, void *Q, uintptr_t stream) {
    if (!plan || !proj || !Q) return FDKOD_ERR_INVALID_ARG;
    return cuda_status(launch_filter(plan->impl, proj, Q, (cudaStream_t)stream));
}

int fdkod_backproject(fdkod_plan_t *plan, const void *Q, float *vol, uintptr_t stream) {
    if (!plan || !Q || !vol) return FDKOD_ERR_INVALID_ARG;
    PlanImpl &p = plan->impl;
    if (p.D > 1 && !p.Sp) return FDKOD_ERR_INVALID_ARG;  // plan made without a workspace
    cudaStream_t st = (cudaStream_t)stream;
    if (p.D == 1) return cuda_status(launch_backproject(p, p.od, true, Q, vol, st));
    FDKOD_TRY(launch_decompose(p, Q, p.Sp, st));
    return cuda_status(launch_backproject(p, p.od, false, p.Sp, vol, st));
}

int fdk_backproject_plain(fdkod_plan_t *plan, const void *Q, float *vol, uintptr_t stream) {
    if (!plan || !Q || !vol) return FDKOD_ERR_INVALID_ARG;
    return cuda_status(launch_backproject(plan->impl, plan->impl.pl, true, Q, vol, (cudaStream_t)stream));
}

int fdkod_decompose(fdkod_plan_t *plan, const void *Q, float *out, uintptr_t stream) {
    if (!plan || !Q || plan->impl.D == 1) return FDKOD_ERR_INVALID_ARG;
    if (!out) out = plan->impl.Sp;  // the plan's own workspace
    if (!out) return FDKOD_ERR_INVALID_ARG;
    return cuda_status(launch_decompose(plan->impl, Q, out, (cudaStream_t)stream));
}

int fdkod_backproject_decomposed(fdkod_plan_t *plan, const float *S, float *vol, uintptr_t stream) {
    if (!plan || !vol || plan->impl.D == 1) return FDKOD_ERR_INVALID_ARG;
    if (!S) S = plan->impl.Sp;  // the plan's own workspace
    if (!S) return FDKOD_ERR_INVALID_ARG;
    return cuda_status(launch_backproject(plan->impl, plan->impl.od, false, S, vol, (cudaStream_t)stream));
}

int fdkod_compute_bounds(fdkod_plan_t *plan, uintptr_t stream) {
    if (!plan) return FDKOD_ERR_INVALID_ARG;
    return cuda_status(launch_bounds(plan->impl, plan->impl.od, (cudaStream_t)stream));
}

int fdkod_get_bounds(const fdkod_plan_t *plan, int32_t *lo, int32_t *hi, int32_t *crop, double *phi,
                     int32_t *w0, int32_t *T) {
    if (!plan) return FDKOD_ERR_INVALID_ARG;
    const PlanImpl &p = plan->impl;
    const size_t n = (size_t)p.od.nsq * p.g.P;
    FDKOD_TRY(cudaDeviceSynchronize());
    if (lo) FDKOD_TRY(cudaMemcpy(lo, p.od.lo, sizeof(int32_t) * n, cudaMemcpyDeviceToHost));
    if (hi) FDKOD_TRY(cudaMemcpy(hi, p.od.hi, sizeof(int32_t) * n, cudaMemcpyDeviceToHost));
    if (crop) FDKOD_TRY(cudaMemcpy(crop, p.od.crop, sizeof(int32_t) * n, cudaMemcpyDeviceToHost));
    if (phi) FDKOD_TRY(cudaMemcpy(phi, p.od.phi, sizeof(double) * n, cudaMemcpyDeviceToHost));
    if (w0) FDKOD_TRY(cudaMemcpy(w0, p.od.w0, sizeof(int32_t) * p.od.nsq, cudaMemcpyDeviceToHost));
    if (T) FDKOD_TRY(cudaMemcpy(T, p.od.T, sizeof(int32_t) * p.od.nsq, cudaMemcpyDeviceToHost));
    return FDKOD_OK;
}

int fdkod_last_device_status(fdkod_plan_t *plan, uintptr_t stream) {
    if (!plan) return FDKOD_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    int h = 0;
    FDKOD_TRY(cudaMemcpyAsync(&h, plan->impl.status, sizeof(int), cudaMemcpyDeviceToHost, st));
    FDKOD_TRY(cudaMemsetAsync(plan->impl.status, 0, sizeof(int), st));
    FDKOD_TRY(cudaStreamSynchronize(st));
    if (h & 2) return FDKOD_ERR_TIMEOUT;
    if (h & 1) return FDKOD_ERR_BOUNDS;
    return FDKOD_OK;
}

int fdkod_slab_rows(const fdkod_plan_t *plan, int z0, int nz, int32_t *v0, int32_t *nrows) {
    if (!plan || !v0 || !nrows) return FDKOD_ERR_INVALID_ARG;
    const fdkod_geometry &g = plan->impl.g;
    if (z0 < 0 || nz < 1 || z0 + nz > g.N) return FDKOD_ERR_INVALID_ARG;
    // U = (R + x cos b + y sin b) / R lies in [1 - r/R, 1 + r/R] for the
    // largest in-slice radius r; the row is z / U + (Nv-1)/2 (Sec. 2.2)
    const double rmax = M_SQRT2 * 0.5 * (double)(g.N - 1);
    const double vc = 0.5 * (double)(g.Nv - 1);
    double lo = INFINITY, hi = -INFINITY;
    const int zs[2] = {z0, z0 + nz - 1};
    for (int i = 0; i < 2; ++i) {
        const double z = (double)zs[i] - 0.5 * (double)(g.N - 1);
        for (double U : {1.0 - rmax / g.R, 1.0 + rmax / g.R}) {
            const double v = z / U + vc;
            lo = fmin(lo, v);
            hi = fmax(hi, v);
        }
    }
    const int a = std::max(0, (int)floor(lo));
    const int b = std::min(g.Nv, (int)floor(hi) + 2);
    *v0 = a;
    *nrows = std::max(1, b - a);
    if (a >= g.Nv) *v0 = g.Nv - 1;
    return FDKOD_OK;
}

int fdkod_filter_rows(fdkod_plan_t *plan, const float *proj_rows, int v0, int nrows, void *Q_rows,
                      uintptr_t stream) {
    if (!plan || !proj_rows || !Q_rows) return FDKOD_ERR_INVALID_ARG;
    const PlanImpl &p = plan->impl;
    if (v0 < 0 || nrows < 1 || v0 + nrows > p.g.Nv) return FDKOD_ERR_INVALID_ARG;
    Band b;
    b.row0 = v0;
    b.nrows = nrows;
    return cuda_status(launch_filter(p, proj_rows, Q_rows, (cudaStream_t)stream, b));
}

int fdkod_backproject_slab(fdkod_plan_t *plan, const void *Q_rows, int v0, int nrows, float *S_work, int z0, int nz,
                           float *vol_slab, uintptr_t stream) {
    if (!plan || !Q_rows || !vol_slab) return FDKOD_ERR_INVALID_ARG;
    PlanImpl &p = plan->impl;
    if (v0 < 0 || nrows < 1 || v0 + nrows > p.g.Nv || z0 < 0 || nz < 1 || z0 + nz > p.g.N)
        return FDKOD_ERR_INVALID_ARG;
    if (p.D > 1 && !S_work) return FDKOD_ERR_INVALID_ARG;
    int32_t need0 = 0, needn = 0;
    fdkod_slab_rows(plan, z0, nz, &need0, &needn);
    if (need0 < v0 || need0 + needn > v0 + nrows) return FDKOD_ERR_INVALID_ARG;  // band misses rows
    Band b;
    b.row0 = v0;
    b.nrows = nrows;
    b.zoff = z0;
    b.nz = nz;
    cudaStream_t st = (cudaStream_t)stream;
    if (p.D == 1) return cuda_status(launch_backproject(p, p.od, true, Q_rows, vol_slab, st, b));
    FDKOD_TRY(launch_decompose(p, Q_rows, S_work, st, b));
    return cuda_status(launch_backproject(p, p.od, false, S_work, vol_slab, st, b));
}

int fdkod_set_decimation_taps(fdkod_plan_t *plan, const double *h, int n) {
    if (!plan || !h) return FDKOD_ERR_INVALID_ARG;
    PlanImpl &p = plan->impl;
    if (p.D < 2 || (n != p.D && n != 2 * p.D)) return FDKOD_ERR_INVALID_ARG;
    for (int i = 0; i < n; ++i)
        if (!std::isfinite(h[i])) return FDKOD_ERR_INVALID_ARG;
    std::vector<float4> w(p.D);
    tap_table(h, n / p.D, p.D, w.data());
    if (cudaMemcpy(p.tapw, w.data(), sizeof(float4) * p.D, cudaMemcpyHostToDevice) != cudaSuccess)
        return FDKOD_ERR_CUDA;
    p.tap_blocks = n / p.D;
    for (int i = 0; i < 2 * fdkod::kMaxTapD; ++i) p.htaps[i] = i < n ? h[i] : 0.0;
    if (p.net && upload_net(p) != cudaSuccess) return FDKOD_ERR_CUDA;
    return FDKOD_OK;
}

int fdkod_get_decimation_taps(const fdkod_plan_t *plan, double *h, int cap) {
    if (!plan || (cap > 0 && !h)) return FDKOD_ERR_INVALID_ARG;
    const PlanImpl &p = plan->impl;
    const int n = p.tap_blocks * p.D;
    for (int i = 0; i < n && i < cap; ++i) h[i] = p.htaps[i];
    return n;
}

int fdkod_sinc_taps(int D, int H, double *h) {
    if (D < 1 || H < 1 || H > 2 || D > fdkod::kMaxTapD || !h) return FDKOD_ERR_INVALID_ARG;
    sinc_taps(D, H, h);
    return FDKOD_OK;
}

int fdkod_set_test_fault(fdkod_plan_t *plan, int kind, int64_t wait_ns) {
    if (!plan || kind < FDKOD_TEST_NONE || kind > FDKOD_TEST_SMALL_WINDOW || wait_ns < 0) return FDKOD_ERR_INVALID_ARG;
    plan->impl.test_fault = kind;
    plan->impl.wait_ns = wait_ns;
    return FDKOD_OK;
}

const char *fdkod_strerror(int status) {
    switch (status) {
        case FDKOD_OK: return "ok";
        case FDKOD_ERR_INVALID_ARG: return "invalid argument";
        case FDKOD_ERR_UNSUPPORTED: return "unsupported configuration";
        case FDKOD_ERR_CUDA: return "CUDA error";
        case FDKOD_ERR_OOM: return "out of memory";
        case FDKOD_ERR_TIMEOUT: return "device wait timed out";
        case FDKOD_ERR_BOUNDS: return "staging window overflow";
    }
    return "unknown status";
}

}  // extern "C"

struct fdkod_batch {
    fdkod::BatchImpl *impl = nullptr;
};

int fdkod_batch_create(fdkod_plan_t *const *plans, const void *const *src, float *const *vols, int count,
                       fdkod_batch_t **out) {
    if (!plans || !vols || !out || count < 1) return FDKOD_ERR_INVALID_ARG;
    *out = nullptr;
    std::vector<const fdkod::PlanImpl *> p((size_t)count);
    std::vector<const void *> s((size_t)count);
    for (int i = 0; i < count; ++i) {
        if (!plans[i] || !vols[i]) return FDKOD_ERR_INVALID_ARG;
        p[i] = &plans[i]->impl;
        s[i] = src ? src[i] : nullptr;
        if (!s[i]) s[i] = p[i]->D > 1 ? (const void *)p[i]->Sp : nullptr;  // the plan's workspace
        if (!s[i]) return FDKOD_ERR_INVALID_ARG;
    }
    bool supported = false;
    fdkod::BatchImpl *b = nullptr;
    const cudaError_t e = fdkod::batch_create(p.data(), s.data(), vols, count, &b, supported);
    if (e != cudaSuccess) return cuda_status(e);
    if (!supported || !b) return FDKOD_ERR_UNSUPPORTED;
    *out = new fdkod_batch{b};
    return FDKOD_OK;
}

int fdkod_batch_backproject(fdkod_batch_t *batch, uintptr_t stream) {
    if (!batch || !batch->impl) return FDKOD_ERR_INVALID_ARG;
    return cuda_status(fdkod::batch_launch(*batch->impl, (cudaStream_t)stream));
}

void fdkod_batch_destroy(fdkod_batch_t *batch) {
    if (!batch) return;
    fdkod::batch_destroy(batch->impl);
    delete batch;
}

namespace {
constexpr int kTileWidths[] = {32, 48, 64, 96, 128};  // the backprojection's instantiated windows
int auto_width(int need) {
    for (int w : kTileWidths)
        if (need <= w) return w;
    return 0;
}
}  // namespace

int fdkod_set_tile(fdkod_plan_t *plan, int window_cols) {
    if (!plan || window_cols < 0) return FDKOD_ERR_INVALID_ARG;
    fdkod::SquareSet &ss = plan->impl.od;
    if (window_cols == 0) {
        ss.WdT = auto_width(ss.need);
        ss.WdT16 = auto_width(ss.need16);
        return FDKOD_OK;
    }
    bool instantiated = false;
    for (int w : kTileWidths) instantiated = instantiated || w == window_cols;
    if (!instantiated || window_cols < ss.need || ss.Rw > 256) return FDKOD_ERR_UNSUPPORTED;
    ss.WdT = window_cols;
    ss.WdT16 = window_cols >= ss.need16 ? window_cols : auto_width(ss.need16);
    return FDKOD_OK;
}

int fdkod_get_tile(const fdkod_plan_t *plan, int *window_cols, int *min_cols) {
    if (!plan) return FDKOD_ERR_INVALID_ARG;
    const fdkod::SquareSet &ss = plan->impl.od;
    if (window_cols) *window_cols = ss.WdT;
    if (min_cols) *min_cols = auto_width(ss.need);
    return FDKOD_OK;
}
