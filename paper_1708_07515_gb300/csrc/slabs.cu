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
