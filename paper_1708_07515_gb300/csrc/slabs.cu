// Whole slab-wise reconstruction from host buffers (piecemeal FDK-OD,
// Sec. 2.2): a three-stream pipeline over z-slabs.  For slab i (buffer
// b = i mod 2) the upload stream copies the detector rows the slab needs,
// from every view, in one strided copy; the compute stream filters those
// rows, decomposes and backprojects the slab; the read-back stream copies
// the slab to the host.  Events order the reuse of the two band and two
// slab buffers, so slab i + 1 uploads while slab i computes and slab i - 1
// downloads.  The filtered rows and the decomposed data are single
// buffers: the compute stream uses them one slab at a time.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <new>
#include <vector>

#include "fdkod_internal.cuh"

namespace fdkod {

// Two band buffers and two slab buffers (double-buffered), the filtered
// rows and the decomposed data of one slab, the upload and read-back
// streams and the per-slab events, made on the first call for a slab size
// and kept with the plan (a call that allocated tens of GB each time spent
// much of its time in cudaMalloc and cudaFree).
struct SlabPipe {
    int slab = 0, nsl = 0;
    std::vector<void *> mem;
    std::vector<cudaEvent_t> ev;
    void *proj_b[2] = {}, *vol_b[2] = {}, *Q = nullptr, *S = nullptr;
    cudaStream_t up = nullptr, down = nullptr;
    int64_t bytes = 0;
    cudaError_t alloc(void **p, size_t n) {
        cudaError_t e = cudaMalloc(p, std::max<size_t>(n, 1));
        if (e == cudaSuccess) {
            mem.push_back(*p);
            bytes += (int64_t)std::max<size_t>(n, 1);
        }
        return e;
    }
};

void free_slab_pipe(SlabPipe *sp) {
    if (!sp) return;
    if (sp->up) cudaStreamSynchronize(sp->up);
    if (sp->down) cudaStreamSynchronize(sp->down);
    for (cudaEvent_t e : sp->ev)
        if (e) cudaEventDestroy(e);
    if (sp->up) cudaStreamDestroy(sp->up);
    if (sp->down) cudaStreamDestroy(sp->down);
    for (void *p : sp->mem) cudaFree(p);
    delete sp;
}

}  // namespace fdkod

namespace {

using fdkod::Band;
using fdkod::PlanImpl;

int status_of(cudaError_t e) {
    if (e == cudaSuccess) return FDKOD_OK;
    return e == cudaErrorMemoryAllocation ? FDKOD_ERR_OOM : FDKOD_ERR_CUDA;
}

#define SLAB_TRY(expr)                         \
    do {                                       \
        const int _rc = status_of(expr);       \
        if (_rc != FDKOD_OK) return _rc;       \
    } while (0)

cudaError_t make_slab_pipe(const PlanImpl &p, int slab, int nsl, int max_rows, fdkod::SlabPipe **out) {
    using fdkod::SlabPipe;
    SlabPipe *sp = new (std::nothrow) SlabPipe;
    if (!sp) return cudaErrorMemoryAllocation;
    const int N = p.g.N, Nu = p.g.Nu, P = p.g.P;
    const size_t es = p.qtype == FDKOD_F32 ? 4 : 2;
    const size_t band = (size_t)P * max_rows * Nu;  // samples of one band of rows
    const size_t vslab = (size_t)slab * N * N;      // voxels of one slab
    cudaError_t e = cudaSuccess;
    for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
        e = sp->alloc(&sp->proj_b[b], sizeof(float) * band);
        if (e == cudaSuccess) e = sp->alloc(&sp->vol_b[b], sizeof(float) * vslab);
    }
    if (e == cudaSuccess) e = sp->alloc(&sp->Q, es * band);
    if (e == cudaSuccess && p.D > 1)
        e = sp->alloc(&sp->S, sizeof(float) * (size_t)p.od.nsq * p.Pd * max_rows * p.Tstride);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&sp->up, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&sp->down, cudaStreamNonBlocking);
    if (e == cudaSuccess) {
        sp->ev.assign(4 * (size_t)nsl, nullptr);
        for (auto &ev : sp->ev)
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    }
    if (e != cudaSuccess) {
        fdkod::free_slab_pipe(sp);
        return e;
    }
    sp->slab = slab;
    sp->nsl = nsl;
    *out = sp;
    return cudaSuccess;
}

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
    if (p.slabs && p.slabs->slab != slab) {  // another slab size: new buffers
        fdkod::free_slab_pipe(p.slabs);
        p.slabs = nullptr;
    }
    if (!p.slabs) {
        fdkod::SlabPipe *sp = nullptr;
        SLAB_TRY(make_slab_pipe(p, slab, nsl, max_rows, &sp));
        p.slabs = sp;
    }
    fdkod::SlabPipe &r = *p.slabs;
    if (device_bytes) *device_bytes = r.bytes;
    void **proj_b = r.proj_b, **vol_b = r.vol_b, *Q = r.Q, *S = r.S;
    cudaEvent_t *ev_up = r.ev.data(), *ev_filt = ev_up + nsl, *ev_comp = ev_filt + nsl, *ev_down = ev_comp + nsl;
    cudaStream_t comp = (cudaStream_t)stream;
    // the previous call's read-backs and the caller's earlier work come first
    SLAB_TRY(cudaEventRecord(ev_comp[0], comp));
    SLAB_TRY(cudaStreamWaitEvent(r.up, ev_comp[0], 0));
    SLAB_TRY(cudaEventRecord(ev_down[0], r.down));
    SLAB_TRY(cudaStreamWaitEvent(comp, ev_down[0], 0));

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
    SLAB_TRY(cudaStreamSynchronize(r.up));
    SLAB_TRY(cudaStreamSynchronize(comp));
    return fdkod_last_device_status(plan, stream);
}

// ---------------------------------------------------------------------------
// Whole-volume reconstruction from host buffers (fdkod_reconstruct): the
// plan keeps device buffers for the projections, the filtered projections
// and the volume, plus an upload and a read-back stream (made on the first
// call).  Within one call
//   - the projections go up in bands of detector rows (every view) on the
//     upload stream, and the compute stream filters and decomposes each band
//     as soon as it has landed (both stages are row-local);
//   - the backprojection runs once every band is decomposed, in groups of
//     slice pairs, and each group's read-back on the read-back stream
//     overlaps the next group's backprojection.
namespace fdkod {

// Row bands of the upload, outside in: two thin outer bands of Nv/8 rows
// (the outermost slice pairs read only those, so their backprojection can
// start early), then bands of Nv/4 rows.  The strided copy of a band (one
// segment per view) keeps near the contiguous copy rate down to about
// 256 KiB segments (measured: 211 GB/s for two bands of 512^2 x 720
// float32, 179 for four, 124 for eight).  A kernel reading a page-locked
// host buffer moves a band at the link's rate whatever its height (207-211
// GB/s), but its CTAs take SM slots from the compute it would overlap: it
// moves only the two outer bands, before any compute has started.
constexpr int kPipeChunks = 8;  // at most this many row bands
constexpr int kPipeSlabs = 16;  // groups of slice pairs of the backprojection / read-back
constexpr int kKernelBands = 2;  // leading bands moved by band_upload_kernel

// Rows v0 .. v0 + nb - 1 of every view (view4 float4 per view, the band at
// float4 offset off4, n4 float4 long) from a host buffer mapped into the
// device's address space to the device copy.  Every index stays below
// P * view4 (off4 + n4 <= view4, checked by the caller).
__global__ void __launch_bounds__(256) band_upload_kernel(const float4 *__restrict__ src, float4 *__restrict__ dst,
                                                          long long view4, long long off4, int n4, int P) {
    for (int k = blockIdx.x; k < P; k += gridDim.x) {
        const float4 *s = src + (long long)k * view4 + off4;
        float4 *d = dst + (long long)k * view4 + off4;
        int j = threadIdx.x;
        // four loads in flight per thread: the link's latency is long
        for (; j + 3 * 256 < n4; j += 4 * 256) {
            const float4 a = s[j], b = s[j + 256], c = s[j + 512], e = s[j + 768];
            d[j] = a;
            d[j + 256] = b;
            d[j + 512] = c;
            d[j + 768] = e;
        }
        for (; j < n4; j += 256) d[j] = s[j];
    }
}

// The bands are filtered and decomposed on a stream of their own (in upload
// order), and the groups' backprojections alternate between the caller's
// stream and a third one: a group fills only part of the GPU, and launches
// on one stream cannot overlap their last partial wave with the next launch.
struct HostPipe {
    float *proj = nullptr, *vol = nullptr;
    void *Q = nullptr;
    cudaStream_t up = nullptr, down = nullptr, comp2 = nullptr, comp3 = nullptr;
    cudaEvent_t ev_up[kPipeChunks] = {}, ev_band[kPipeChunks] = {}, ev_slab[kPipeSlabs] = {};
    cudaEvent_t ev_start = nullptr, ev_join = nullptr;
    int64_t bytes = 0;
    int sms = 1;  // CTAs of a band upload
};

void free_host_pipe(HostPipe *hp) {
    if (!hp) return;
    if (hp->up) cudaStreamSynchronize(hp->up);
    if (hp->down) cudaStreamSynchronize(hp->down);
    if (hp->comp2) cudaStreamSynchronize(hp->comp2);
    if (hp->comp3) cudaStreamSynchronize(hp->comp3);
    for (cudaEvent_t e : hp->ev_up)
        if (e) cudaEventDestroy(e);
    for (cudaEvent_t e : hp->ev_band)
        if (e) cudaEventDestroy(e);
    for (cudaEvent_t e : hp->ev_slab)
        if (e) cudaEventDestroy(e);
    if (hp->ev_start) cudaEventDestroy(hp->ev_start);
    if (hp->ev_join) cudaEventDestroy(hp->ev_join);
    if (hp->up) cudaStreamDestroy(hp->up);
    if (hp->down) cudaStreamDestroy(hp->down);
    if (hp->comp2) cudaStreamDestroy(hp->comp2);
    if (hp->comp3) cudaStreamDestroy(hp->comp3);
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
    int dev = 0;
    cudaError_t e;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess ||
        (e = cudaDeviceGetAttribute(&hp->sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess ||
        (e = cudaMalloc(&hp->proj, sizeof(float) * samples)) != cudaSuccess ||
        (e = cudaMalloc(&hp->Q, es * samples)) != cudaSuccess ||
        (e = cudaMalloc(&hp->vol, sizeof(float) * voxels)) != cudaSuccess ||
        (e = cudaStreamCreateWithFlags(&hp->up, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaStreamCreateWithFlags(&hp->down, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaStreamCreateWithFlags(&hp->comp2, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaStreamCreateWithFlags(&hp->comp3, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&hp->ev_start, cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&hp->ev_join, cudaEventDisableTiming)) != cudaSuccess) {
        fdkod::free_host_pipe(hp);
        return e;
    }
    for (cudaEvent_t *evs : {hp->ev_up, hp->ev_band})
        for (int i = 0; i < fdkod::kPipeChunks; ++i)
            if ((e = cudaEventCreateWithFlags(&evs[i], cudaEventDisableTiming)) != cudaSuccess) {
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

// The device address of host buffer p of `bytes` bytes when the GPU can read
// all of it directly -- page-locked memory mapped into the device's address
// space (cudaHostAlloc, cudaHostRegister) whose allocation covers the whole
// buffer, 16-byte aligned -- else nullptr (pageable memory, a buffer that
// runs past its allocation, or a driver that does not say).
const void *mapped_host_source(const void *p, size_t bytes) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();  // not sticky: clear it
        return nullptr;
    }
    if (a.type != cudaMemoryTypeHost || !a.devicePointer || ((uintptr_t)a.devicePointer & 15u)) return nullptr;
    static const PFN_cuPointerGetAttribute_v4000 get = [] {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuPointerGetAttribute", &fn, 4000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess) {
            cudaGetLastError();
            return (PFN_cuPointerGetAttribute_v4000) nullptr;
        }
        return (PFN_cuPointerGetAttribute_v4000)fn;
    }();
    if (!get) return nullptr;
    const CUdeviceptr dp = (CUdeviceptr)(uintptr_t)a.devicePointer;
    CUdeviceptr start = 0;
    size_t size = 0;
    if (get(&start, CU_POINTER_ATTRIBUTE_RANGE_START_ADDR, dp) != CUDA_SUCCESS ||
        get(&size, CU_POINTER_ATTRIBUTE_RANGE_SIZE, dp) != CUDA_SUCCESS)
        return nullptr;
    if (dp < start || dp - start > size || bytes > size - (size_t)(dp - start)) return nullptr;
    return a.devicePointer;
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
    cudaStream_t comp = (cudaStream_t)stream;
    // the previous call's work on the compute stream (and the caller's) comes first
    SLAB_TRY(cudaEventRecord(hp.ev_start, comp));
    SLAB_TRY(cudaStreamWaitEvent(hp.up, hp.ev_start, 0));
    SLAB_TRY(cudaStreamWaitEvent(hp.comp2, hp.ev_start, 0));
    SLAB_TRY(cudaStreamWaitEvent(hp.comp3, hp.ev_start, 0));
    cudaStream_t cs[2] = {comp, hp.comp3};  // backprojection groups
    // upload in bands of detector rows (every view, one strided copy per
    // band), outermost bands first; the filter and the decomposition are
    // row-local, so each band is filtered and decomposed as soon as it has
    // landed.  A slice pair (p, N - 1 - p) reads rows near both edges of the
    // detector (row z/U + (Nv-1)/2, Sec. 2.2), so the outermost pairs can be
    // backprojected once the two outer bands are done, while the inner bands
    // are still on their way.  Bands hold an even number of rows from an even
    // first row (the filter pairs rows in one complex transform, as the
    // whole-detector launch does); an odd Nv, or a learned decimation (its
    // kernel takes every row at once), makes one band.
    const bool banded = (Nv % 2) == 0 && !p.net;
    // band i covers rows bv[i] .. bv[i + 1] - 1 (even bounds); upload order:
    // the two outer bands, then inwards, alternating bottom and top
    int bv[kPipeChunks + 1], nbands = 0;
    if (!banded) {
        bv[0] = 0;
        bv[1] = Nv;
        nbands = 1;
    } else {
        const int outer = std::max(2, (Nv / 8) & ~1), inner = std::max(2, (Nv / 4) & ~1);
        int lo = 0, hi = Nv, cuts_lo[kPipeChunks], cuts_hi[kPipeChunks], nl = 0, nh = 0;
        for (int step = outer; lo < hi; step = inner) {  // walk inwards from both ends
            if (nl + nh + 2 > kPipeChunks - 1 || hi - lo <= 2 * step) break;
            lo += step;
            hi -= step;
            cuts_lo[nl++] = lo;
            cuts_hi[nh++] = hi;
        }
        bv[nbands++] = 0;
        for (int i = 0; i < nl; ++i) bv[nbands++] = cuts_lo[i];
        for (int i = nh - 1; i >= 0; --i) bv[nbands++] = cuts_hi[i];
        bv[nbands] = Nv;  // nbands = number of bands
    }
    int order[kPipeChunks];  // outside in: 0, last, 1, last - 1, ...
    for (int i = 0, lo = 0, hi = nbands - 1; i < nbands; ++i) order[i] = (i & 1) ? hi-- : lo++;
    // the two outer bands from a host buffer the GPU can read: a kernel (the
    // GPU has no other work yet); every other band: strided copy-engine
    // transfers
    const void *mapped = (Nu % 4) == 0 ? mapped_host_source(proj_host, sizeof(float) * view * (size_t)P) : nullptr;
    const size_t pitch = sizeof(float) * view;
    for (int i = 0; i < nbands; ++i) {
        const int v0 = bv[order[i]], nb = bv[order[i] + 1] - v0;
        if (mapped && i < fdkod::kKernelBands) {
            // float4 units: a view is Nv Nu / 4 of them, the band starts v0 Nu / 4 in
            fdkod::band_upload_kernel<<<std::max(1, std::min(P, hp.sms)), 256, 0, hp.up>>>(
                (const float4 *)mapped, (float4 *)hp.proj, (long long)(view / 4), (long long)v0 * Nu / 4,
                nb * Nu / 4, P);
            SLAB_TRY(cudaGetLastError());
        } else {
            SLAB_TRY(cudaMemcpy2DAsync(hp.proj + (size_t)v0 * Nu, pitch, proj_host + (size_t)v0 * Nu, pitch,
                                       sizeof(float) * (size_t)nb * Nu, (size_t)P, cudaMemcpyHostToDevice,
                                       hp.up));
        }
        SLAB_TRY(cudaEventRecord(hp.ev_up[order[i]], hp.up));
    }
    SLAB_TRY(fdkod::launch_bounds(p, p.od, comp));
    SLAB_TRY(cudaEventRecord(hp.ev_join, comp));
    SLAB_TRY(cudaStreamWaitEvent(hp.comp2, hp.ev_join, 0));  // the bounds before any decomposition
    for (int i = 0; i < nbands; ++i) {
        const int bi = order[i];
        fdkod::Band rows;
        rows.row0 = bv[bi];
        rows.nrows = bv[bi + 1] - bv[bi];
        rows.whole_arrays = true;
        cudaStream_t c = hp.comp2;
        SLAB_TRY(cudaStreamWaitEvent(c, hp.ev_up[bi], 0));
        SLAB_TRY(fdkod::launch_filter(p, hp.proj, hp.Q, c, rows));
        if (p.D > 1 && banded) SLAB_TRY(fdkod::launch_decompose(p, hp.Q, p.Sp, c, rows));
        SLAB_TRY(cudaEventRecord(hp.ev_band[bi], c));
    }
    if (p.D > 1 && !banded) {
        SLAB_TRY(fdkod::launch_decompose(p, hp.Q, p.Sp, hp.comp2));
        SLAB_TRY(cudaEventRecord(hp.ev_band[0], hp.comp2));
    }
    // make stream c wait for the bands holding detector rows that slices
    // z0 .. z0 + nz - 1 can read (the bound of fdkod_slab_rows)
    auto wait_rows = [&](cudaStream_t c, int z0, int nz) -> int {
        int32_t v0 = 0, nr = 0;
        const int rc = fdkod_slab_rows(plan, z0, nz, &v0, &nr);
        if (rc != FDKOD_OK) return rc;
        for (int bi = 0; bi < nbands; ++bi)
            if (bv[bi] < v0 + nr && bv[bi + 1] > v0) SLAB_TRY(cudaStreamWaitEvent(c, hp.ev_band[bi], 0));
        return FDKOD_OK;
    };
    const bool direct = p.D == 1;
    const void *src = direct ? hp.Q : (const void *)p.Sp;
    // backprojection in groups of slice pairs (slices p and N - 1 - p, the
    // same tiles as one whole-volume launch), outermost first, alternating
    // between the two compute streams, each after the bands it reads; each
    // group's two z-ranges are read back as soon as it is done
    const int npair = (N + 1) / 2;
    int ps = (npair + kPipeSlabs - 1) / kPipeSlabs;
    ps = (ps + fdkod::kZP - 1) / fdkod::kZP * fdkod::kZP;
    int ns = 0;
    bool paired = true;
    const size_t plane = (size_t)N * N;
    for (int pa = 0; pa < npair && paired; pa += ps, ++ns) {
        const int pb = std::min(pa + ps, npair);
        cudaStream_t c = cs[ns & 1];
        int rc = wait_rows(c, pa, pb - pa);
        if (rc == FDKOD_OK) rc = wait_rows(c, N - pb, pb - pa);
        if (rc != FDKOD_OK) return rc;
        SLAB_TRY(fdkod::launch_backproject_pairs(p, p.od, direct, src, hp.vol, c, pa, pb, paired));
        if (!paired) break;  // not staged: z-slabs below (before anything was launched)
        SLAB_TRY(cudaEventRecord(hp.ev_slab[ns], c));
        SLAB_TRY(cudaStreamWaitEvent(hp.down, hp.ev_slab[ns], 0));
        SLAB_TRY(cudaMemcpyAsync(vol_host + (size_t)pa * plane, hp.vol + (size_t)pa * plane,
                                 sizeof(float) * (size_t)(pb - pa) * plane, cudaMemcpyDeviceToHost, hp.down));
        const int u0 = std::max(N - pb, pb), u1 = N - pa;  // upper slices, the middle one (odd N) once
        if (u1 > u0)
            SLAB_TRY(cudaMemcpyAsync(vol_host + (size_t)u0 * plane, hp.vol + (size_t)u0 * plane,
                                     sizeof(float) * (size_t)(u1 - u0) * plane, cudaMemcpyDeviceToHost, hp.down));
    }
    if (!paired)  // the z-slab fallback reads every band
        for (int bi = 0; bi < nbands; ++bi) {
            SLAB_TRY(cudaStreamWaitEvent(comp, hp.ev_band[bi], 0));
            SLAB_TRY(cudaStreamWaitEvent(hp.comp3, hp.ev_band[bi], 0));
        }
    // z-slabs of whole 32-slice tiles where the staged pair kernel does not apply
    int zs = (N + kPipeSlabs - 1) / kPipeSlabs;
    zs = (zs + fdkod::kZT - 1) / fdkod::kZT * fdkod::kZT;
    if (!paired) ns = 0;
    for (int z0 = 0; z0 < N && !paired; z0 += zs, ++ns) {
        fdkod::Band b;
        b.zoff = z0;
        b.nz = std::min(zs, N - z0);
        float *dst = hp.vol + (size_t)z0 * plane;
        cudaStream_t c = cs[ns & 1];
        SLAB_TRY(fdkod::launch_backproject(p, p.od, direct, src, dst, c, b));
        SLAB_TRY(cudaEventRecord(hp.ev_slab[ns], c));
        SLAB_TRY(cudaStreamWaitEvent(hp.down, hp.ev_slab[ns], 0));
        SLAB_TRY(cudaMemcpyAsync(vol_host + (size_t)z0 * plane, dst, sizeof(float) * (size_t)b.nz * plane,
                                 cudaMemcpyDeviceToHost, hp.down));
    }
    SLAB_TRY(cudaStreamSynchronize(hp.comp2));
    SLAB_TRY(cudaStreamSynchronize(hp.comp3));
    SLAB_TRY(cudaStreamSynchronize(hp.down));
    SLAB_TRY(cudaStreamSynchronize(comp));
    return fdkod_last_device_status(plan, stream);
}
