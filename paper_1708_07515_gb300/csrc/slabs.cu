// Whole slab-wise reconstruction from host buffers (piecemeal FDK-OD,
// Sec. 2.2): a three-stream pipeline over z-slabs.  For slab i (buffer
// b = i mod 2) the upload stream copies the detector rows the slab needs,
// from every view, in one strided copy; the compute stream filters those
// rows, decomposes and backprojects the slab; the read-back stream copies
// the slab to the host.  Events order the reuse of the two band and two
// slab buffers, so slab i + 1 uploads while slab i computes and slab i - 1
// downloads.  The filtered rows and the decomposed data are single
// buffers: the compute stream uses them one slab at a time.
#include <cuda_runtime.h>

#include <algorithm>
#include <new>
#include <vector>

#include "fdkod_internal.cuh"

namespace {

using fdkod::Band;
using fdkod::PlanImpl;

struct Resources {
    std::vector<void *> mem;
    std::vector<cudaEvent_t> ev;
    cudaStream_t up = nullptr, down = nullptr;
    int64_t bytes = 0;
    ~Resources() {
        if (up) cudaStreamSynchronize(up);
        if (down) cudaStreamSynchronize(down);
        for (cudaEvent_t e : ev) cudaEventDestroy(e);
        if (up) cudaStreamDestroy(up);
        if (down) cudaStreamDestroy(down);
        for (void *p : mem) cudaFree(p);
    }
    cudaError_t alloc(void **p, size_t n) {
        cudaError_t e = cudaMalloc(p, std::max<size_t>(n, 1));
        if (e == cudaSuccess) {
            mem.push_back(*p);
            bytes += (int64_t)std::max<size_t>(n, 1);
        }
        return e;
    }
};

int status_of(cudaError_t e) {
    if (e == cudaSuccess) return FDKOD_OK;
    return e == cudaErrorMemoryAllocation ? FDKOD_ERR_OOM : FDKOD_ERR_CUDA;
}

#define SLAB_TRY(expr)                         \
    do {                                       \
        const int _rc = status_of(expr);       \
        if (_rc != FDKOD_OK) return _rc;       \
    } while (0)

}  // namespace

extern "C" int fdkod_reconstruct_slabs(fdkod_plan_t *plan, const float *proj_host, float *vol_host, int slab,
                                       uintptr_t stream, int64_t *device_bytes) {
    if (!plan || !proj_host || !vol_host || slab < 1) return FDKOD_ERR_INVALID_ARG;
    PlanImpl &p = plan->impl;
    const int N = p.g.N, Nv = p.g.Nv, Nu = p.g.Nu, P = p.g.P;
    slab = std::min(slab, N);
    const int nsl = (N + slab - 1) / slab;
    std::vector<int32_t> z0(nsl), nz(nsl), v0(nsl), nr(nsl);
    int max_rows = 1;
    for (int i = 0; i < nsl; ++i) {
        z0[i] = i * slab;
        nz[i] = std::min(slab, N - z0[i]);
        const int rc = fdkod_slab_rows(plan, z0[i], nz[i], &v0[i], &nr[i]);
        if (rc != FDKOD_OK) return rc;
        max_rows = std::max(max_rows, (int)nr[i]);
    }
    const size_t es = p.qtype == FDKOD_F32 ? 4 : 2;
    const size_t band = (size_t)P * max_rows * Nu;  // samples of one band of rows
    const size_t vslab = (size_t)slab * N * N;      // voxels of one slab

    Resources r;
    void *proj_b[2], *vol_b[2], *Q = nullptr, *S = nullptr;
    for (int b = 0; b < 2; ++b) {
        SLAB_TRY(r.alloc(&proj_b[b], sizeof(float) * band));
        SLAB_TRY(r.alloc(&vol_b[b], sizeof(float) * vslab));
    }
    SLAB_TRY(r.alloc(&Q, es * band));
    if (p.D > 1) SLAB_TRY(r.alloc(&S, sizeof(float) * (size_t)p.od.nsq * p.Pd * max_rows * p.Tstride));
    if (device_bytes) *device_bytes = r.bytes;
    SLAB_TRY(cudaStreamCreateWithFlags(&r.up, cudaStreamNonBlocking));
    SLAB_TRY(cudaStreamCreateWithFlags(&r.down, cudaStreamNonBlocking));
    r.ev.assign(4 * (size_t)nsl, nullptr);
    for (auto &e : r.ev) SLAB_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    cudaEvent_t *ev_up = r.ev.data(), *ev_filt = ev_up + nsl, *ev_comp = ev_filt + nsl, *ev_down = ev_comp + nsl;
    cudaStream_t comp = (cudaStream_t)stream;

    for (int i = 0; i < nsl; ++i) {
        const int b = i & 1;
        // upload: rows v0 .. v0 + nr - 1 of every view, once the filter of
        // slab i - 2 has read this band buffer
        if (i >= 2) SLAB_TRY(cudaStreamWaitEvent(r.up, ev_filt[i - 2], 0));
        const size_t row_bytes = sizeof(float) * (size_t)nr[i] * Nu;
        SLAB_TRY(cudaMemcpy2DAsync(proj_b[b], row_bytes, proj_host + (size_t)v0[i] * Nu, sizeof(float) * (size_t)Nv * Nu,
                                   row_bytes, (size_t)P, cudaMemcpyHostToDevice, r.up));
        SLAB_TRY(cudaEventRecord(ev_up[i], r.up));
        // compute
        SLAB_TRY(cudaStreamWaitEvent(comp, ev_up[i], 0));
        Band rows;
        rows.row0 = v0[i];
        rows.nrows = nr[i];
        SLAB_TRY(fdkod::launch_filter(p, (const float *)proj_b[b], Q, comp, rows));
        SLAB_TRY(cudaEventRecord(ev_filt[i], comp));
        if (i >= 2) SLAB_TRY(cudaStreamWaitEvent(comp, ev_down[i - 2], 0));  // slab buffer read back
        Band sl = rows;
        sl.zoff = z0[i];
        sl.nz = nz[i];
        if (p.D == 1) {
            SLAB_TRY(fdkod::launch_backproject(p, p.od, true, Q, (float *)vol_b[b], comp, sl));
        } else {
            SLAB_TRY(fdkod::launch_decompose(p, Q, (float *)S, comp, sl));
            SLAB_TRY(fdkod::launch_backproject(p, p.od, false, S, (float *)vol_b[b], comp, sl));
        }
        SLAB_TRY(cudaEventRecord(ev_comp[i], comp));
        // read back
        SLAB_TRY(cudaStreamWaitEvent(r.down, ev_comp[i], 0));
        SLAB_TRY(cudaMemcpyAsync(vol_host + (size_t)z0[i] * N * N, vol_b[b], sizeof(float) * (size_t)nz[i] * N * N,
                                 cudaMemcpyDeviceToHost, r.down));
        SLAB_TRY(cudaEventRecord(ev_down[i], r.down));
    }
    SLAB_TRY(cudaStreamSynchronize(r.down));
    SLAB_TRY(cudaStreamSynchronize(comp));
    return fdkod_last_device_status(plan, stream);
}

// ---------------------------------------------------------------------------
// Whole-volume reconstruction from host buffers (fdkod_reconstruct): the
// plan keeps device buffers for the projections, the filtered projections
// and the volume, plus an upload and a read-back stream (made on the first
// call).  Within one call
//   - the projections go up in chunks of views on the upload stream, and
//     the compute stream filters each chunk as soon as it has landed;
//   - the bounds, the decomposition and the backprojection run on the
//     compute stream once every view is filtered;
//   - the backprojection runs in z-slabs, and each slab's read-back on the
//     read-back stream overlaps the next slab's backprojection.
namespace fdkod {

constexpr int kPipeChunks = 8;  // view chunks of the upload
constexpr int kPipeSlabs = 4;   // z-slabs of the backprojection / read-back

struct HostPipe {
    float *proj = nullptr, *vol = nullptr;
    void *Q = nullptr;
    cudaStream_t up = nullptr, down = nullptr;
    cudaEvent_t ev_up[kPipeChunks] = {}, ev_slab[kPipeSlabs] = {}, ev_start = nullptr;
    int64_t bytes = 0;
};

void free_host_pipe(HostPipe *hp) {
    if (!hp) return;
    if (hp->up) cudaStreamSynchronize(hp->up);
    if (hp->down) cudaStreamSynchronize(hp->down);
    for (cudaEvent_t e : hp->ev_up)
        if (e) cudaEventDestroy(e);
    for (cudaEvent_t e : hp->ev_slab)
        if (e) cudaEventDestroy(e);
    if (hp->ev_start) cudaEventDestroy(hp->ev_start);
    if (hp->up) cudaStreamDestroy(hp->up);
    if (hp->down) cudaStreamDestroy(hp->down);
    cudaFree(hp->proj);
    cudaFree(hp->Q);
    cudaFree(hp->vol);
    delete hp;
}

}  // namespace fdkod

namespace {

cudaError_t make_pipe(PlanImpl &p, fdkod::HostPipe **out) {
    using fdkod::HostPipe;
    HostPipe *hp = new (std::nothrow) HostPipe;
    if (!hp) return cudaErrorMemoryAllocation;
    const size_t samples = (size_t)p.g.P * p.g.Nv * p.g.Nu;
    const size_t es = p.qtype == FDKOD_F32 ? 4 : 2;
    const size_t voxels = (size_t)p.g.N * p.g.N * p.g.N;
    cudaError_t e;
    if ((e = cudaMalloc(&hp->proj, sizeof(float) * samples)) != cudaSuccess ||
        (e = cudaMalloc(&hp->Q, es * samples)) != cudaSuccess ||
        (e = cudaMalloc(&hp->vol, sizeof(float) * voxels)) != cudaSuccess ||
        (e = cudaStreamCreateWithFlags(&hp->up, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaStreamCreateWithFlags(&hp->down, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&hp->ev_start, cudaEventDisableTiming)) != cudaSuccess) {
        fdkod::free_host_pipe(hp);
        return e;
    }
    for (auto &ev : hp->ev_up)
        if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess) {
            fdkod::free_host_pipe(hp);
            return e;
        }
    for (auto &ev : hp->ev_slab)
        if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess) {
            fdkod::free_host_pipe(hp);
            return e;
        }
    hp->bytes = (int64_t)(sizeof(float) * samples + es * samples + sizeof(float) * voxels);
    *out = hp;
    return cudaSuccess;
}

}  // namespace

extern "C" int fdkod_reconstruct(fdkod_plan_t *plan, const float *proj_host, float *vol_host, uintptr_t stream) {
    using fdkod::kPipeChunks;
    using fdkod::kPipeSlabs;
    if (!plan || !proj_host || !vol_host) return FDKOD_ERR_INVALID_ARG;
    PlanImpl &p = plan->impl;
    if (p.D > 1 && !p.Sp) return FDKOD_ERR_INVALID_ARG;  // plan made without a workspace
    if (!p.pipe) {
        fdkod::HostPipe *hp = nullptr;
        SLAB_TRY(make_pipe(p, &hp));
        p.pipe = hp;
        p.device_bytes += hp->bytes;
    }
    fdkod::HostPipe &hp = *p.pipe;
    const int N = p.g.N, Nv = p.g.Nv, Nu = p.g.Nu, P = p.g.P;
    const size_t view = (size_t)Nv * Nu;
    const size_t es = p.qtype == FDKOD_F32 ? 4 : 2;
    cudaStream_t comp = (cudaStream_t)stream;
    // the previous call's work on the compute stream (and the caller's) comes first
    SLAB_TRY(cudaEventRecord(hp.ev_start, comp));
    SLAB_TRY(cudaStreamWaitEvent(hp.up, hp.ev_start, 0));
    // upload in chunks of an even number of views (the filter pairs rows in
    // one complex transform; even chunk starts keep the whole-array pairing)
    int cv = (P + kPipeChunks - 1) / kPipeChunks;
    cv += cv & 1;
    int nch = 0;
    for (int k0 = 0; k0 < P; k0 += cv, ++nch) {
        const int nv = std::min(cv, P - k0);
        SLAB_TRY(cudaMemcpyAsync(hp.proj + (size_t)k0 * view, proj_host + (size_t)k0 * view,
                                 sizeof(float) * view * nv, cudaMemcpyHostToDevice, hp.up));
        SLAB_TRY(cudaEventRecord(hp.ev_up[nch], hp.up));
    }
    SLAB_TRY(fdkod::launch_bounds(p, p.od, comp));
    nch = 0;
    for (int k0 = 0; k0 < P; k0 += cv, ++nch) {
        const int nv = std::min(cv, P - k0);
        SLAB_TRY(cudaStreamWaitEvent(comp, hp.ev_up[nch], 0));
        SLAB_TRY(fdkod::launch_filter(p, hp.proj + (size_t)k0 * view, (char *)hp.Q + es * (size_t)k0 * view, comp,
                                      fdkod::Band{}, nv));
    }
    if (p.D > 1) SLAB_TRY(fdkod::launch_decompose(p, hp.Q, p.Sp, comp));
    const bool direct = p.D == 1;
    const void *src = direct ? hp.Q : (const void *)p.Sp;
    // backprojection in groups of slice pairs (slices p and N - 1 - p, the
    // same tiles as one whole-volume launch); each group's two z-ranges are
    // read back while the next group is computed
    const int npair = (N + 1) / 2;
    int ps = (npair + kPipeSlabs - 1) / kPipeSlabs;
    ps = (ps + fdkod::kZP - 1) / fdkod::kZP * fdkod::kZP;
    int ns = 0;
    bool paired = true;
    for (int pa = 0; pa < npair && paired; pa += ps, ++ns) {
        const int pb = std::min(pa + ps, npair);
        SLAB_TRY(fdkod::launch_backproject_pairs(p, p.od, direct, src, hp.vol, comp, pa, pb, paired));
        if (!paired) break;  // not staged: z-slabs below (before anything was launched)
        SLAB_TRY(cudaEventRecord(hp.ev_slab[ns], comp));
        SLAB_TRY(cudaStreamWaitEvent(hp.down, hp.ev_slab[ns], 0));
        const size_t plane = (size_t)N * N;
        SLAB_TRY(cudaMemcpyAsync(vol_host + (size_t)pa * plane, hp.vol + (size_t)pa * plane,
                                 sizeof(float) * (size_t)(pb - pa) * plane, cudaMemcpyDeviceToHost, hp.down));
        const int u0 = std::max(N - pb, pb), u1 = N - pa;  // upper slices, the middle one (odd N) once
        if (u1 > u0)
            SLAB_TRY(cudaMemcpyAsync(vol_host + (size_t)u0 * plane, hp.vol + (size_t)u0 * plane,
                                     sizeof(float) * (size_t)(u1 - u0) * plane, cudaMemcpyDeviceToHost, hp.down));
    }
    // z-slabs of whole 32-slice tiles where the staged pair kernel does not apply
    int zs = (N + kPipeSlabs - 1) / kPipeSlabs;
    zs = (zs + fdkod::kZT - 1) / fdkod::kZT * fdkod::kZT;
    if (!paired) ns = 0;
    for (int z0 = 0; z0 < N && !paired; z0 += zs, ++ns) {
        fdkod::Band b;
        b.zoff = z0;
        b.nz = std::min(zs, N - z0);
        float *dst = hp.vol + (size_t)z0 * N * N;
        SLAB_TRY(fdkod::launch_backproject(p, p.od, direct, src, dst, comp, b));
        SLAB_TRY(cudaEventRecord(hp.ev_slab[ns], comp));
        SLAB_TRY(cudaStreamWaitEvent(hp.down, hp.ev_slab[ns], 0));
        SLAB_TRY(cudaMemcpyAsync(vol_host + (size_t)z0 * N * N, dst, sizeof(float) * (size_t)b.nz * N * N,
                                 cudaMemcpyDeviceToHost, hp.down));
    }
    SLAB_TRY(cudaStreamSynchronize(hp.down));
    SLAB_TRY(cudaStreamSynchronize(comp));
    return fdkod_last_device_status(plan, stream);
}
