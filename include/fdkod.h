/*
 * fdkod.h -- C ABI of the GB300 (sm_103a) FDK-OD cone-beam backprojection
 * library, libfdkod.so.
 *
 * Method: Andriiashen & Kozhevnikov, "Fast optimal decomposed modification
 * of FDK with potential decreasing of memory consuming" (2017).  FDK
 * filters each detector row and backprojects every voxel as a weighted sum
 * of P samples (Sec. 1, Sec. 2.1).  FDK-OD splits every slice into 4^s
 * squares of side N/2^s (Sec. 2.2), bounds the detector columns each square
 * needs per view with Eq. 1 at the square's vertices (Sec. 2.1), shifts the
 * cropped rows so the square centre sits on one column, low-pass filters
 * and downsamples them along the view axis by D (angular decimation,
 * Sec. 2.1), and backprojects each square from the P/D remaining views.
 *
 * Conventions (shared by every entry point):
 *  - lengths in voxels; voxel centres x_i = i - (N-1)/2 (same for y, z);
 *  - views beta_k = 2 pi k / P, k = 0..P-1, over a full orbit; source at
 *    -R (cos beta, sin beta, 0); R is the source-to-isocentre distance
 *    that appears in Eq. 1;
 *  - virtual flat detector through the isocentre with unit pitch, columns
 *    u = 0..Nu-1, rows v = 0..Nv-1, a = u - (Nu-1)/2, b = v - (Nv-1)/2;
 *  - projections proj[P][Nv][Nu] float32 (u fastest), filtered projections
 *    Q[P][Nv][Nu] in the plan's storage type, volume vol[N][N][N] float32
 *    indexed [z][y][x] (x fastest);
 *  - every device pointer is a CUDA device address owned by the caller;
 *    the library never frees or retains it after the call returns;
 *  - `stream` is a cudaStream_t passed as an integer (0 = legacy default
 *    stream); all device work of a call is enqueued on it and the call
 *    returns without waiting, except where a function says it synchronises;
 *  - there is no CPU fallback: every compute step runs in CUDA kernels.
 *
 * Errors: every int-returning function returns FDKOD_OK (0) or a negative
 * fdkod_status; no function throws or aborts.  Asynchronous kernel faults
 * surface as FDKOD_ERR_CUDA on a later call.  Kernels that detect an
 * out-of-window access record it in a per-plan device status word instead
 * of trapping; fdkod_last_device_status() reads and clears it.
 */
#ifndef FDKOD_H
#define FDKOD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    FDKOD_OK = 0,
    FDKOD_ERR_INVALID_ARG = -1, /* null pointer, non-positive size, bad enum */
    FDKOD_ERR_UNSUPPORTED = -2, /* D does not divide P, 2^s > N, source inside the volume, sizes over limits */
    FDKOD_ERR_CUDA = -3,        /* a CUDA runtime call or kernel launch failed */
    FDKOD_ERR_OOM = -4,         /* device or host allocation failed */
    FDKOD_ERR_TIMEOUT = -5,     /* a bounded device-side wait gave up */
    FDKOD_ERR_BOUNDS = -6       /* a kernel's staging window was too small (result invalid) */
} fdkod_status;

/* Storage type of the filtered projections Q. */
typedef enum { FDKOD_F32 = 0, FDKOD_BF16 = 1, FDKOD_F16 = 2 } fdkod_dtype;

/* Circular-orbit cone-beam geometry (Sec. 2.1; R as in Eq. 1). */
typedef struct {
    double R;   /* source-to-isocentre distance, voxels; must exceed the volume's half-diagonal + 1 */
    int32_t N;  /* volume is N x N x N voxels */
    int32_t Nu; /* detector columns */
    int32_t Nv; /* detector rows */
    int32_t P;  /* views over 360 degrees */
} fdkod_geometry;

typedef struct fdkod_plan fdkod_plan_t;

/* Read-only facts about a plan (sizes of its internal buffers). */
typedef struct {
    int32_t s, D, Pd;        /* decomposition level, decimation factor, P/D */
    int32_t n_squares;       /* 4^s */
    int32_t T_stride;        /* row stride (elements) of the decomposed data */
    int32_t fft_length;      /* FFT length of the filter stage */
    int64_t decomposed_elems;/* n_squares * Pd * Nv * T_stride (0 when D == 1) */
    int64_t device_bytes;    /* device memory the plan holds */
} fdkod_plan_info;

/*
 * Build a plan for geometry *g, decomposition level s (4^s squares of side
 * N/2^s, Sec. 2.2) and decimation factor D (P/D views per square after the
 * angular decimation of Sec. 2.1; D = 1 means crop only, which equals plain
 * FDK).  qtype is the storage type fdkod_filter writes and the
 * backprojections read.
 *
 * Computes, on the device in FP64, the per-(square, view) crop bounds of
 * Eq. 1 at the square vertices, the shift centres and the shifted-row
 * windows, and allocates the decomposed-data workspace.  Synchronises the
 * device before returning.  On success *out owns all plan memory; release
 * it with fdkod_destroy.  Errors: INVALID_ARG (null g/out, non-positive
 * sizes, R <= 0, unknown qtype), UNSUPPORTED (P % D != 0, s < 0,
 * s > 7, 2^s > N, R not beyond the volume, sizes above 2^15, Nu above
 * 8192), OOM, CUDA.
 */
int fdkod_plan(const fdkod_geometry *g, int s, int D, fdkod_dtype qtype, fdkod_plan_t **out);

/* Flags of fdkod_plan_ex. */
#define FDKOD_PLAN_NO_WORKSPACE 1 /* do not allocate the whole-volume decomposed-data workspace */
#define FDKOD_PLAN_SINC_TAPS 2    /* windowed-sinc angular low-pass instead of the triangle */

/*
 * fdkod_plan with flags.  FDKOD_PLAN_NO_WORKSPACE leaves out the
 * 4^s * (P/D) * Nv * T_stride float workspace of fdkod_backproject: such a
 * plan serves the slab-wise entry points below (piecemeal reconstruction,
 * Sec. 2.2), and fdkod_backproject then returns FDKOD_ERR_INVALID_ARG when
 * D > 1.  FDKOD_PLAN_SINC_TAPS selects the Hann-windowed sinc of
 * fdkod_sinc_taps with H = 2 as the angular low-pass of the decomposition
 * (Sec. 2.1 leaves the filter open; the default is the triangle
 * (D - |i|) / D^2, |i| < D).  Other flags: INVALID_ARG.  Otherwise as
 * fdkod_plan; D above 128 is UNSUPPORTED.
 */
int fdkod_plan_ex(const fdkod_geometry *g, int s, int D, fdkod_dtype qtype, int flags, fdkod_plan_t **out);

/* Release a plan (NULL is ignored).  Waits for the device to finish. */
void fdkod_destroy(fdkod_plan_t *plan);

/* Fill *info.  Errors: INVALID_ARG. */
int fdkod_get_info(const fdkod_plan_t *plan, fdkod_plan_info *info);

/*
 * FDK filter stage (Sec. 1; the "initial convolution" of Sec. 3): for every
 * detector row, q = proj * R / sqrt(R^2 + a^2 + b^2), then linear
 * convolution along u with the discrete Ram-Lak kernel (h(0) = 1/4,
 * h(n odd) = -1/(pi^2 n^2), h(n even) = 0), zero outside the detector.
 * proj: device [P][Nv][Nu] float32.  Q: device [P][Nv][Nu] of the plan's
 * qtype.  proj and Q must not overlap.  Errors: INVALID_ARG, CUDA.
 */
int fdkod_filter(fdkod_plan_t *plan, const float *proj, void *Q, uintptr_t stream);

/*
 * FDK-OD backprojection (Sec. 2.2): vol = for every square, the sum over
 * the P/D decimated views beta_{jD} of U^-2 times the bilinear sample of
 * the decomposed data at column t = u - phi - w0 and row z/U + (Nv-1)/2,
 * scaled by pi / (P/D).  For D > 1 the decomposed data is first built in
 * the plan's workspace (shift by linear interpolation, triangle low-pass
 * (D-|i|)/D^2 circular over views, downsample by D; Sec. 2.1).  D = 1
 * reads each square's crop of Q directly.  Q: device [P][Nv][Nu] qtype;
 * vol: device [N][N][N] float32, fully overwritten.  Concurrent calls with
 * the same plan race on its workspace.  Errors: INVALID_ARG, CUDA.
 */
int fdkod_backproject(fdkod_plan_t *plan, const void *Q, float *vol, uintptr_t stream);

/*
 * Plain FDK backprojection (Sec. 2.1, the baseline of the speedup):
 * vol = (pi/P) sum_k U_k^-2 Q_k(u, v) over all P views with bilinear
 * interpolation, u from Eq. 1 and v = z/U + (Nv-1)/2.  Same arguments,
 * layouts and errors as fdkod_backproject.
 */
int fdk_backproject_plain(fdkod_plan_t *plan, const void *Q, float *vol, uintptr_t stream);

/*
 * The decomposition stage on its own (Sec. 2.1 shift + angular
 * decimation): writes S'[q][j][v][t] (float32, t < T_stride, zero for
 * t >= T[q]) for all squares q, decimated views j < P/D and rows v to the
 * device buffer out of info.decomposed_elems floats, or, with out NULL, to
 * the plan's own workspace (the one fdkod_backproject uses; the batched
 * backprojection reads it).  Errors: INVALID_ARG (also when D == 1, or out
 * NULL for a plan without a workspace), CUDA.
 */
int fdkod_decompose(fdkod_plan_t *plan, const void *Q, float *out, uintptr_t stream);

/*
 * Backprojection stage of FDK-OD on its own: the same sum as
 * fdkod_backproject for D > 1, reading decomposed data S (device, the
 * layout fdkod_decompose writes) instead of the plan's workspace.  With
 * fdkod_decompose it splits fdkod_backproject into its two kernels, e.g.
 * to time them apart.  S NULL reads the plan's own workspace.  Errors:
 * INVALID_ARG (also when D == 1, or S NULL without a workspace), CUDA.
 */
int fdkod_backproject_decomposed(fdkod_plan_t *plan, const float *S, float *vol, uintptr_t stream);

/*
 * Recompute the plan's per-(square, view) bounds, shift centres and
 * backprojection coefficients on the device (Eq. 1 at the vertices,
 * FP64), asynchronously on `stream`, without allocating and without host
 * synchronisation.  The plan computes them once at creation; this entry
 * point exists so a pipeline step can include the bound stage.  The
 * results are identical to the plan's.  Errors: INVALID_ARG, CUDA.
 */
int fdkod_compute_bounds(fdkod_plan_t *plan, uintptr_t stream);

/*
 * Piecemeal reconstruction (Sec. 2.2: FDK-OD needs only the part of the
 * sinogram its part of the image uses).  A slab of slices z0 .. z0+nz-1
 * reads only the detector rows the row formula b = z R / (R + x cos b +
 * y sin b) can reach; these three calls let a caller hold just those rows,
 * the slab's decomposed data and the slab's volume on the device.
 *
 * fdkod_slab_rows: the band [*v0, *v0 + *nrows) of detector rows slices
 * z0 .. z0+nz-1 need (host arithmetic, no device work).  Errors:
 * INVALID_ARG (null, empty or out-of-range slab).
 */
int fdkod_slab_rows(const fdkod_plan_t *plan, int z0, int nz, int32_t *v0, int32_t *nrows);

/*
 * fdkod_filter_rows: the filter of fdkod_filter on detector rows
 * v0 .. v0+nrows-1 only.  proj_rows, Q_rows: device [P][nrows][Nu] (float32,
 * plan's qtype).  Errors: INVALID_ARG (also for a band outside the
 * detector), CUDA.
 */
int fdkod_filter_rows(fdkod_plan_t *plan, const float *proj_rows, int v0, int nrows, void *Q_rows,
                      uintptr_t stream);

/*
 * fdkod_backproject_slab: fdkod_backproject restricted to slices
 * z0 .. z0+nz-1, reading filtered rows v0 .. v0+nrows-1 only.  Q_rows:
 * device [P][nrows][Nu] of the plan's qtype; S_work: device float
 * workspace of n_squares * Pd * nrows * T_stride elements (fdkod_get_info;
 * unused, may be NULL, when D == 1); vol_slab: device [nz][N][N] float32,
 * fully overwritten.  The band must contain the rows fdkod_slab_rows
 * returns for the slab.  Errors: INVALID_ARG (null pointers, slab or band
 * out of range, band missing needed rows, no S_work with D > 1), CUDA.
 */
int fdkod_backproject_slab(fdkod_plan_t *plan, const void *Q_rows, int v0, int nrows, float *S_work, int z0,
                           int nz, float *vol_slab, uintptr_t stream);

/*
 * Copy the plan's crop bounds to host arrays (each may be NULL):
 * lo, hi, crop [4^s][P] int32 (lo = floor(min u) and hi = floor(max u) + 1
 * over the square's four vertex voxel centres, so linear interpolation at
 * any voxel of the square reads columns lo..hi; crop = floor(phi + w0),
 * the first column the shifted row reads); phi [4^s][P] float64, the column of
 * the square centre's projection; w0, T [4^s] int32, the offset and width
 * of the shifted rows (sample t sits at column phi + w0 + t).  Synchronises
 * the device.  Errors: INVALID_ARG, CUDA.
 */
int fdkod_get_bounds(const fdkod_plan_t *plan, int32_t *lo, int32_t *hi, int32_t *crop,
                     double *phi, int32_t *w0, int32_t *T);

/*
 * Read and clear the plan's device status word after the work queued on
 * `stream` (synchronises the stream).  Returns FDKOD_OK, FDKOD_ERR_BOUNDS
 * (a staging window overflowed; the affected output is invalid),
 * FDKOD_ERR_TIMEOUT, or FDKOD_ERR_CUDA.
 */
int fdkod_last_device_status(fdkod_plan_t *plan, uintptr_t stream);

/*
 * FDK-OD backprojection that allocates nothing.  The paper has no
 * counterpart: this is a deployment variant of fdkod_backproject.
 *
 * For callers that cannot call cudaMalloc, e.g. an acquisition pipeline
 * that fixes its device memory at start-up and forbids allocation later
 * (cudaMalloc may synchronise the device and its latency is unbounded), or
 * a host application whose own memory pool has already reserved the
 * device, so an extra cudaMalloc would fail.  It needs no plan: it computes
 * the bounds, the decomposed data and the volume of fdkod_plan(g, s, D,
 * FDKOD_F32) + fdkod_backproject in one call, with the same kernels.
 *
 * Working memory: one file-scope device array of 48 MiB inside libfdkod,
 * which every GPU that loads the library holds until the process exits.
 * A call needs 52 bytes per (square, view) pair plus 4 * 4^s * (P/D) * Nv
 * * T_stride bytes of decomposed data (T_stride ~ 1.4 N/2^s + 8) plus a few
 * KiB; larger problems return FDKOD_ERR_UNSUPPORTED without touching the
 * GPU.  Example: 128^3 from 128 views, s = 2, D = 2 needs about 30 MiB.
 *
 * First call on a device: with that device current, the call looks up the
 * array's device address (cudaGetSymbolAddress).  With lazy module loading
 * this is also when the driver loads the library's device code and reserves
 * the array, which may synchronise the device, or fail with FDKOD_ERR_CUDA
 * when the device has no room left.  Make one warm-up call per device at
 * start-up.
 *
 * Every call shares the array and it keeps the previous call's contents:
 * the call clears what must start at zero, but calls whose work overlaps on
 * the GPU (other streams, other host threads without ordering) race on it --
 * order them on one stream.  Host callers are serialised by a mutex.  The
 * call's tables (view cos/sin, low-pass weights) are computed on the device:
 * it copies nothing from host memory and does not wait for the stream.
 * Device-side checks (a staging window or a shifted-row width too small, a
 * bounded wait that gave up) set the array's status word, which
 * fdkod_noalloc_device_status reads; this call itself returns FDKOD_OK once
 * the work is enqueued.
 *
 * g, s, D: as fdkod_plan; Q: device [P][Nv][Nu] float32 (already
 * filtered); vol: device [N][N][N] float32, fully overwritten; work is
 * enqueued on `stream`.  Errors: INVALID_ARG, UNSUPPORTED (as fdkod_plan,
 * P > 8192, or over the 48 MiB limit), CUDA.
 */
int fdkod_backproject_noalloc(const fdkod_geometry *g, int s, int D, const float *Q, float *vol,
                              uintptr_t stream);

/*
 * Device status of the most recent fdkod_backproject_noalloc call on the
 * current device (the paper has no counterpart): waits for the work queued
 * on `stream`, then reads and clears the status word of the fixed array
 * (allocates nothing).  Returns FDKOD_OK, FDKOD_ERR_BOUNDS (a staging window
 * or the host bound of the shifted-row width was too small: the volume is
 * invalid), FDKOD_ERR_TIMEOUT (a bounded device-side wait gave up), or
 * FDKOD_ERR_CUDA.
 */
int fdkod_noalloc_device_status(uintptr_t stream);

/*
 * Whole reconstruction from host buffers: the FDK filter (Sec. 1), the bound
 * computation of Eq. 1 and the FDK-OD backprojection (Sec. 2.2) of one scan,
 * from projections in host memory to a volume in host memory.
 *
 * proj_host: host [P][Nv][Nu] float32; vol_host: host [N][N][N] float32,
 * fully overwritten.  Page-locked host memory lets the copies overlap the
 * compute; pageable memory works, with synchronous copies.  Within the call
 * the projections are uploaded in bands of detector rows and each band is
 * filtered and decomposed as soon as it has landed (both stages are
 * row-local); the volume is then backprojected in groups of slices and each
 * group is copied back while the next one is computed (an upload and a
 * read-back stream of the plan's own, ordered after the work already queued
 * on `stream`).  When proj_host is page-locked memory mapped into the
 * device's address space (cudaHostAlloc, cudaHostRegister; one allocation
 * holding all of it, 16-byte aligned, Nu a multiple of 4), a kernel reads
 * the two outer bands from it directly; copy-engine transfers move every
 * other band.  The volume equals fdkod_filter + fdkod_backproject bit for
 * bit when Nv is even (for odd Nv the filter pairs rows differently: equal
 * to float32 round-off).
 * Device memory: the first call allocates, and the plan then keeps until
 * fdkod_destroy, buffers for the projections, the filtered projections and
 * the volume (reported in fdkod_plan_info.device_bytes); the plan must have
 * its decomposed-data workspace when D > 1.  Synchronous: returns once
 * vol_host holds the volume and the device status word has been read.
 * Calls with the same plan must not overlap.  Errors: INVALID_ARG (null
 * pointers, a plan without a workspace and D > 1), OOM, CUDA, TIMEOUT,
 * BOUNDS.
 */
int fdkod_reconstruct(fdkod_plan_t *plan, const float *proj_host, float *vol_host, uintptr_t stream);

/*
 * Whole slab-wise reconstruction from host buffers (piecemeal FDK-OD,
 * Sec. 2.2): the device holds two bands of detector rows and two slabs at a
 * time, never the whole projection set or volume.  Per slab of `slab`
 * slices: one strided copy uploads, from every view, the detector rows the
 * slab needs (fdkod_slab_rows); the filter, decomposition and backprojection
 * run on `stream`; the slab is copied back.  Uploads and read-backs run on
 * streams of their own, double-buffered, so they overlap the neighbouring
 * slabs' compute.
 *
 * proj_host: host [P][Nv][Nu] float32 (page-locked memory lets the copies
 *   overlap the compute; pageable memory works, with synchronous copies);
 * vol_host: host [N][N][N] float32, fully overwritten;
 * slab: slices per slab (>= 1, clamped to N);
 * device_bytes: if not NULL, receives the device memory of the slab
 *   pipeline (band and slab buffers, filtered rows, decomposed data).  The
 *   first call for a slab size allocates it; it stays with the plan for
 *   later calls with the same slab size (another size replaces it) and is
 *   freed by fdkod_destroy.  It is not counted in fdkod_plan_info.
 * Works with plans with or without the whole-volume workspace; the plan's
 * decimation taps and storage type apply.  Synchronous: returns once
 * vol_host holds the volume and the device status word has been read.
 * Errors: INVALID_ARG, OOM, CUDA, TIMEOUT, BOUNDS.
 */
int fdkod_reconstruct_slabs(fdkod_plan_t *plan, const float *proj_host, float *vol_host, int slab,
                            uintptr_t stream, int64_t *device_bytes);

/*
 * Angular low-pass of the decomposition (Sec. 2.1: low-pass filter over the
 * angles, then keep every D-th).  The filter is symmetric and circular over
 * the orbit: decimated view j is sum_i h[|i|] S[(jD + i) mod P], |i| < n,
 * with n = D (support of the triangle) or n = 2D.
 *
 * fdkod_set_decimation_taps: copy h[0 .. n-1] (host, not retained) into
 *   the plan; n must be D or 2D and the plan must have D > 1.  Synchronous;
 *   call it while no launch of this plan is in flight.  The taps are used as
 *   given (scale them to unit sum for unit gain).  Errors: INVALID_ARG
 *   (n, D, non-finite values), CUDA.
 * fdkod_get_decimation_taps: the plan's n taps into h[0 .. min(n, cap)-1];
 *   returns n (>= 1) or INVALID_ARG.
 * fdkod_sinc_taps: host only, no device work: the Hann-windowed sinc with
 *   its cutoff at the decimated Nyquist frequency pi / D,
 *   g_i = sinc(i / D) (1 + cos(pi i / (H D))) / 2 for |i| < H D, scaled to
 *   unit sum, into h[0 .. H D - 1].  H is 1 or 2.  Errors: INVALID_ARG
 *   (D < 1 or above 128, H outside 1..2, h NULL).
 */
int fdkod_set_decimation_taps(fdkod_plan_t *plan, const double *h, int n);
int fdkod_get_decimation_taps(const fdkod_plan_t *plan, double *h, int cap);
int fdkod_sinc_taps(int D, int H, double *h);

/*
 * Learned angular decimation (Sec. 2.1 leaves the low-pass open and says
 * its implementation sets the quality).  With a net set, the decomposition
 * of fdkod_backproject, fdkod_decompose and the slab-wise entry points makes
 * each decimated view the plain low-pass above plus a residual network
 * along the view axis, applied to every shifted column (v, t) of a square
 * as a circular sequence x[k] over the orbit (C = 16 channels, 5 taps at
 * offsets m - 2, cross-correlation, no biases):
 *   a1[c][k] = max(0, sum_m W1[c][m] x[k+m-2])
 *   a2[c][k] = max(0, sum_{c',m} W2[c][c'][m] a1[c'][k+m-2])
 *   S'[j]   += sum_{c,m} W3[c][m] a2[c][jD+m-2]
 * Weights: FDKOD_NET_SIZE floats, W1 [16][5], then W2 [16][16][5] (output
 * channel, input channel, tap), then W3 [16][5].  Inference stores them as
 * BF16 (round to nearest even), rounds each layer's input (x, a1, a2) to
 * BF16 and accumulates in FP32; all three layers run on the tensor cores.
 *
 * fdkod_set_decimation_net: copy w (host, not retained) into the plan; w
 *   NULL removes the net (plain low-pass again).  Synchronous; call it
 *   while no launch of this plan is in flight.  Errors: INVALID_ARG (n !=
 *   FDKOD_NET_SIZE, non-finite values), UNSUPPORTED (D < 2 or D > 60),
 *   OOM, CUDA.
 * fdkod_get_decimation_net: the plan's BF16-rounded weights as floats into
 *   w[0 .. min(FDKOD_NET_SIZE, cap)-1]; returns FDKOD_NET_SIZE, or 0 when
 *   no net is set.
 *
 * Training support (FP32, asynchronous on `stream`, device pointers):
 * fdkod_net_adjoint: the adjoint of the FDK-OD backprojection of decomposed
 *   data (Sec. 2.2), one slice z: with e = vol_slice - ref_slice ([N][N],
 *   y then x), adds to dS ([4^s][P/D][Nv][T_stride], the layout of
 *   fdkod_decompose) for every voxel and decimated view j the term
 *   (pi / (P/D)) U^-2 e times the bilinear weight of the sample the
 *   backprojection reads, and adds sum e^2 to *sq_err.  dS then holds
 *   the gradient of (1/2) sum e^2 with respect to the decomposed data.
 * fdkod_net_backward: for detector rows row_lo .. row_hi - 1, recompute the
 *   net's forward pass from Q (all rows, qtype) with the FP32 weights w
 *   (device, FDKOD_NET_SIZE floats) and add to dW (device, same layout) the
 *   gradient of sum dS . S' (dS as above, the gradient of the decimated
 *   views).  Errors of both: INVALID_ARG (null pointers, z or rows out of
 *   range, D < 2), UNSUPPORTED (D > 60), CUDA.
 */
#define FDKOD_NET_SIZE 1440
int fdkod_set_decimation_net(fdkod_plan_t *plan, const float *w, int n);
int fdkod_get_decimation_net(const fdkod_plan_t *plan, float *w, int cap);
int fdkod_net_adjoint(fdkod_plan_t *plan, const float *vol_slice, const float *ref_slice, int z, float *dS,
                      float *sq_err, uintptr_t stream);
int fdkod_net_backward(fdkod_plan_t *plan, const void *Q, const float *w, const float *dS, int row_lo,
                       int row_hi, float *dW, uintptr_t stream);

/*
 * Batched backprojection (the batched form): many plans' FDK-OD
 * backprojections in one persistent launch.  fdkod_batch_create records, per
 * plan i, its source src[i] (device; D = 1: Q, float32 [P][Nv][Nu]; D > 1:
 * decomposed data [4^s][P/D][Nv][T_stride] as fdkod_decompose writes it, or
 * NULL for the plan's own workspace, which fdkod_decompose fills when its
 * out is NULL) and volume vols[i] (device, [N][N][N]); it builds one tensor
 * map per plan and a work list of (plan, tile, z-slab) items, largest plans
 * first, on the device (synchronous; the batch keeps pointers, not copies:
 * the plans and buffers must outlive it).  fdkod_batch_backproject resets
 * the work counter and launches one kernel of as many CTAs as the GPU
 * holds; each takes items until none are left (asynchronous on `stream`,
 * no allocation: it can be captured into a CUDA graph).  The result equals
 * each plan's fdkod_backproject_decomposed / fdkod_backproject of the same
 * source.  Device-side status (window overflow, wait timeout) goes to each
 * plan's status word (fdkod_last_device_status).  Errors: INVALID_ARG (null
 * pointers, count < 1, NULL source for a plan without one), UNSUPPORTED (a
 * plan with 16-bit Q and D = 1, or windows that no TMA box holds: use the
 * per-plan entry points), OOM, CUDA.
 */
typedef struct fdkod_batch fdkod_batch_t;
int fdkod_batch_create(fdkod_plan_t *const *plans, const void *const *src, float *const *vols, int count,
                       fdkod_batch_t **out);
int fdkod_batch_backproject(fdkod_batch_t *batch, uintptr_t stream);
void fdkod_batch_destroy(fdkod_batch_t *batch);

/*
 * Tile shape of the FDK-OD backprojection (for an autotuner): each CTA
 * stages, per view, a window of the source covering its 16 x 16 x 32-voxel
 * tile's footprint; the window width (columns) is one of the instantiated
 * 32, 48, 64, 96, 128.  By default a plan takes the narrowest one that holds
 * every tile's footprint.  fdkod_set_tile(plan, cols) selects a wider one
 * (cols = 0: back to the default); results are the same bit for bit, only
 * the shared-memory layout (bank conflicts) and occupancy change.
 * fdkod_get_tile returns the width in use (float32 windows) and the
 * narrowest valid one (0 when no window fits: the unstaged kernels run).
 * Call while no launch of the plan is in flight.  Errors: INVALID_ARG,
 * UNSUPPORTED (a width that is not instantiated or too narrow).
 */
int fdkod_set_tile(fdkod_plan_t *plan, int window_cols);
int fdkod_get_tile(const fdkod_plan_t *plan, int *window_cols, int *min_cols);

/*
 * Test hooks of the device-side failure paths (the paper has no
 * counterpart; for tests of the error reporting, no GPU fault involved).
 * They act on this plan's staged (TMA) backprojection launches only.
 *  FDKOD_TEST_NONE: no hook (the default).
 *  FDKOD_TEST_SKIP_COPY: the first CTA of a launch leaves out one staging
 *    copy of its second chunk of views, so that chunk's bounded wait runs
 *    out: the CTA records FDKOD_ERR_TIMEOUT, waits (bounded) for its other
 *    copies in flight and exits; the other CTAs finish normally.  Needs more
 *    than 4 backprojected views to act.
 *  FDKOD_TEST_SMALL_WINDOW: every staged window counts as too small, so
 *    every view is skipped (nothing is read outside a window) and
 *    FDKOD_ERR_BOUNDS is recorded.
 * wait_ns: limit of the bounded waits of those launches (0 = the default,
 * 2 s), so a test does not wait seconds.  Volumes written while a hook is
 * set are invalid.  Call while no launch of the plan is in flight.
 * Errors: INVALID_ARG (null plan, unknown kind, negative wait_ns).
 */
#define FDKOD_TEST_NONE 0
#define FDKOD_TEST_SKIP_COPY 1
#define FDKOD_TEST_SMALL_WINDOW 2
int fdkod_set_test_fault(fdkod_plan_t *plan, int kind, int64_t wait_ns);

/* Static message for a status code. */
const char *fdkod_strerror(int status);

#ifdef __cplusplus
}
#endif

#endif /* FDKOD_H */
