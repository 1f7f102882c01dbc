// fdkod_backproject_noalloc: the FDK-OD backprojection without any device
// (or host heap) allocation, for callers that cannot call cudaMalloc -- for
// example an acquisition pipeline that fixes its device memory at start-up
// and forbids allocation afterwards (cudaMalloc can synchronise the device
// and has unbounded latency), or a host application whose own pool has
// already reserved the device memory, so that an extra cudaMalloc fails.
//
// All working memory of the call -- view cos/sin, per-(square, view) bounds
// and coefficients, the status word and the decomposed data S' -- lives in
// one file-scope device array of kScratchBytes.  Every GPU that loads the
// library holds that array until the process exits.  The caller passes Q
// and vol, as for fdkod_backproject.  The call's tables are computed by a
// kernel on the device, so it copies nothing from host memory (nothing
// that a later call could overwrite before the copy runs, and no wait for
// the stream's earlier work).
#include <math.h>
#include <string.h>

#include <algorithm>
#include <mutex>

#include "fdkod_internal.cuh"

namespace {

constexpr size_t kScratchBytes = 48u << 20;  // 48 MiB
constexpr int kMaxDevices = 64;
constexpr int kMaxViews = 8192;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_mutex;
void *g_scratch_addr[kMaxDevices] = {};
double2 g_cs_host[kMaxViews];  // host cos/sin for the host-side sizing (under g_mutex)

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

double centre(int i, int n) { return (double)i - 0.5 * (double)(n - 1); }

void square_range(int q, int m, int N, int &i0, int &i1) {
    i0 = (int)(((long long)q * N + m - 1) / m);
    i1 = (int)((((long long)q + 1) * N + m - 1) / m) - 1;
}

// Host upper bound of max_q T[q] (the device computes the exact widths):
// the same FP64 expressions as the bound kernel, plus one column of slack.
int max_width(const fdkod_geometry &g, int s, const double2 *cs) {
    const int m = 1 << s;
    const double uc = 0.5 * (double)(g.Nu - 1);
    int tmax = 0;
    for (int q = 0; q < m * m; ++q) {
        int ix0, ix1, iy0, iy1;
        square_range(q % m, m, g.N, ix0, ix1);
        square_range(q / m, m, g.N, iy0, iy1);
        const double xs[2] = {centre(ix0, g.N), centre(ix1, g.N)};
        const double ys[2] = {centre(iy0, g.N), centre(iy1, g.N)};
        const double xc = 0.5 * (xs[0] + xs[1]), yc = 0.5 * (ys[0] + ys[1]);
        double dmin = INFINITY, dmax = -INFINITY;
        for (int k = 0; k < g.P; ++k) {
            const double cb = cs[k].x, sb = cs[k].y;
            const double p = g.R * (yc * cb - xc * sb) / (g.R + xc * cb + yc * sb) + uc;
            for (int a = 0; a < 2; ++a)
                for (int b = 0; b < 2; ++b) {
                    const double u = g.R * (ys[b] * cb - xs[a] * sb) / (g.R + xs[a] * cb + ys[b] * sb) + uc;
                    dmin = fmin(dmin, u - p);
                    dmax = fmax(dmax, u - p);
                }
        }
        const int w = (int)floor(dmin) - 1;
        const int T = (int)floor(dmax) + 3 - w + 1;
        if (T > tmax) tmax = T;
    }
    return tmax;
}

// Per-call tables on the device: the status word (cleared), cos/sin of
// every view (the planned path's formula, evaluated in FP64 on the device)
// and the running-sum weights of the triangle low-pass, view j D + r adding
// (D - r) / D^2 to decimated view j and r / D^2 to view j + 1.
__global__ void noalloc_tables_kernel(int P, int D, double2 *cs, float4 *tapw, int *status) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) *status = 0;
    if (i < P) {
        const double beta = 2.0 * M_PI * (double)i / (double)P;
        cs[i] = make_double2(cos(beta), sin(beta));
    }
    if (i < D) {
        const double dd = (double)D * (double)D;
        tapw[i] = make_float4((float)((double)(D - i) / dd), i == 0 ? 0.f : (float)((double)i / dd), 0.f, 0.f);
    }
}

// The decomposed rows are Tstride wide (a host bound); a square whose exact
// width T (from the bound kernel) exceeds it would lose columns: report it
// as a window overflow.
__global__ void noalloc_width_check_kernel(const int32_t *T, int nsq, int Tstride, int *status) {
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nsq; q += gridDim.x * blockDim.x)
        if (T[q] > Tstride) atomicOr(status, 1);
}

// The array's device address on the current device (looked up once per
// device, under g_mutex); null when the lookup fails.
unsigned char *scratch_base() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return nullptr;
    if (!g_scratch_addr[dev]) {
        // host code cannot use g_scratch's name as a device address: ask the
        // runtime for this device's copy, once, with the device current
        void *ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_scratch) != cudaSuccess || !ptr) return nullptr;
        g_scratch_addr[dev] = ptr;
    }
    return (unsigned char *)g_scratch_addr[dev];
}

}  // namespace

extern "C" int fdkod_backproject_noalloc(const fdkod_geometry *g, int s, int D, const float *Q, float *vol,
                                         uintptr_t stream) {
    using namespace fdkod;
    if (!g || !Q || !vol) return FDKOD_ERR_INVALID_ARG;
    if (!(g->R > 0.0) || g->N <= 0 || g->Nu <= 0 || g->Nv <= 0 || g->P <= 0 || D <= 0) return FDKOD_ERR_INVALID_ARG;
    if (g->N > (1 << 15) || g->Nu > (1 << 15) || g->Nv > (1 << 15) || g->P > kMaxViews) return FDKOD_ERR_UNSUPPORTED;
    if (s < 0 || s > 7 || (1 << s) > g->N || g->P % D != 0 || D > fdkod::kMaxTapD) return FDKOD_ERR_UNSUPPORTED;
    if (!(g->R > M_SQRT2 * 0.5 * (double)g->N + 1.0)) return FDKOD_ERR_UNSUPPORTED;

    std::lock_guard<std::mutex> lock(g_mutex);
    unsigned char *base = scratch_base();
    if (!base) return FDKOD_ERR_CUDA;

    PlanImpl p;
    p.g = *g;
    p.s = s;
    p.D = D;
    p.Pd = g->P / D;
    p.qtype = FDKOD_F32;
    for (int k = 0; k < g->P; ++k) {
        const double beta = 2.0 * M_PI * (double)k / (double)g->P;
        g_cs_host[k] = make_double2(cos(beta), sin(beta));
    }
    SquareSet &ss = p.od;
    ss.s = s;
    ss.m = 1 << s;
    ss.nsq = ss.m * ss.m;
    const size_t n = (size_t)ss.nsq * g->P;
    ss.Tmax = max_width(*g, s, g_cs_host);
    p.Tstride = (ss.Tmax + 3) & ~3;
    p.sp_elems = D > 1 ? (int64_t)ss.nsq * p.Pd * g->Nv * p.Tstride : 0;

    // carve the scratch array; reject what does not fit
    size_t off = 0;
    auto take = [&](size_t bytes) {
        unsigned char *ptr = base + off;
        off = align256(off + bytes);
        return ptr;
    };
    p.status = (int *)take(sizeof(int));  // first: fdkod_noalloc_device_status reads it here
    p.cs = (double2 *)take(sizeof(double2) * g->P);
    ss.lo = (int32_t *)take(sizeof(int32_t) * n);
    ss.hi = (int32_t *)take(sizeof(int32_t) * n);
    ss.crop = (int32_t *)take(sizeof(int32_t) * n);
    ss.phi = (double *)take(sizeof(double) * n);
    ss.geo = (GeomEntry *)take(sizeof(GeomEntry) * n);
    ss.w0 = (int32_t *)take(sizeof(int32_t) * ss.nsq);
    ss.T = (int32_t *)take(sizeof(int32_t) * ss.nsq);
    p.tapw = (float4 *)take(sizeof(float4) * (size_t)D);
    p.Sp = (float *)take(sizeof(float) * (size_t)p.sp_elems);
    if (off > kScratchBytes) return FDKOD_ERR_UNSUPPORTED;
    size_windows(p, ss, g_cs_host);

    cudaStream_t st = (cudaStream_t)stream;
    // the array keeps the previous call's contents: the table kernel clears
    // the status word; every other region is fully rewritten below before it
    // is read
    const int nt = std::max(g->P, D);
    noalloc_tables_kernel<<<(nt + 255) / 256, 256, 0, st>>>(g->P, D, p.cs, p.tapw, p.status);
    if (cudaGetLastError() != cudaSuccess) return FDKOD_ERR_CUDA;
    if (launch_bounds(p, ss, st) != cudaSuccess) return FDKOD_ERR_CUDA;
    if (D == 1) return launch_backproject(p, ss, true, Q, vol, st) == cudaSuccess ? FDKOD_OK : FDKOD_ERR_CUDA;
    noalloc_width_check_kernel<<<1, 256, 0, st>>>(ss.T, ss.nsq, p.Tstride, p.status);
    if (cudaGetLastError() != cudaSuccess) return FDKOD_ERR_CUDA;
    if (launch_decompose(p, Q, p.Sp, st) != cudaSuccess) return FDKOD_ERR_CUDA;
    return launch_backproject(p, ss, false, p.Sp, vol, st) == cudaSuccess ? FDKOD_OK : FDKOD_ERR_CUDA;
}

extern "C" int fdkod_noalloc_device_status(uintptr_t stream) {
    std::lock_guard<std::mutex> lock(g_mutex);
    unsigned char *base = scratch_base();
    if (!base) return FDKOD_ERR_CUDA;
    int *status = (int *)base;  // the first region of every call's layout
    cudaStream_t st = (cudaStream_t)stream;
    int h = 0;
    if (cudaMemcpyAsync(&h, status, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemsetAsync(status, 0, sizeof(int), st) != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess)
        return FDKOD_ERR_CUDA;
    if (h & 2) return FDKOD_ERR_TIMEOUT;
    if (h & 1) return FDKOD_ERR_BOUNDS;
    return FDKOD_OK;
}
