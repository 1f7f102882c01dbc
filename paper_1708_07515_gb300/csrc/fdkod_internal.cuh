// Internal declarations shared by the CUDA translation units of libfdkod.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include "../../include/fdkod.h"

namespace fdkod {

// Per-(square, view) backprojection geometry, from FP64 values computed by
// the bound kernel.  With (dx, dy) a voxel's offset from the square centre
// (x_c, y_c) and d_c = R + x_c cos b + y_c sin b:
//   g = R / d_c (1/U at the centre), stored as an unevaluated float pair
//       g_hi + g_lo so the row origin z_c g keeps FP64-level accuracy,
//   r = 1 / d_c,  e = a_c / R,  alpha = -sin b - e cos b,  gamma = cos b - e sin b,
//   1/U = g / (1 + r (cb dx + sb dy)),
//   a(x, y) - a(x_c, y_c) = (1/U) (alpha dx + gamma dy)      (Eq. 1 rearranged),
// so the kernels work with small square-local numbers in FP32.
// frac = (phi + w0) - floor(phi + w0), the sub-pixel part of the shift.
struct GeomEntry {
    float g_hi, g_lo;
    float cb, sb, r, alpha, gamma, frac;
};
static_assert(sizeof(GeomEntry) == 32, "GeomEntry layout");

// One decomposition of the slice into m x m squares (m = 2^s) with its
// per-square, per-view tables on the device.
struct SquareSet {
    int s = 0, m = 1, nsq = 1;
    int32_t *lo = nullptr, *hi = nullptr, *crop = nullptr, *w0 = nullptr, *T = nullptr;
    double *phi = nullptr;
    GeomEntry *geo = nullptr;
    int32_t Tmax = 0;
    // staging window of the backprojection kernel (elements), from a host
    // FP64 sweep over every tile and view; WdT is the width of the TMA path
    // (4-element alignment slack, rounded up to a kernel instantiation, 0
    // when no instantiation is wide enough)
    int Wd = 0, Rw = 0, WdT = 0, WdT16 = 0;  // WdT16: the same for 16-bit windows
    int Rw2 = 0;  // rows of a window of kZP slices (the mirrored-pair kernel)
    int need = 0, need16 = 0;  // the narrowest TMA windows that hold every tile's footprint
    int tiles_per_side = 1;  // 16-voxel tiles per square side
};

constexpr int kTile = 16;      // tile side in x and y (threads per CTA = 256)
constexpr int kZT = 32;        // z voxels per thread
constexpr int kZP = 16;        // slices per half of the mirrored-pair kernel (2 kZP voxels per thread)
constexpr int kViewsPerChunk = 8;  // generic backprojection kernel
constexpr int kViewsPerStage = 4;  // TMA backprojection kernel (two stages)
constexpr int kMaxTapD = 128;      // largest decimation factor with a tap table

// learned angular decimation: 16 channels, 5 taps, 1440 weights
constexpr int kNetChannels = 16, kNetTaps = 5;
constexpr int kNetSize = kNetChannels * kNetTaps * (kNetChannels + 2);
constexpr int kNetMaxD = 60;  // one output view per 64-view chunk needs D <= 60
// Device copy of the learned decimation's weights, BF16-rounded, as the
// tensor-core B operands (16 x 16, K-major, two 8-value planes of 256 bytes):
// layer 2 per tap m (output x input channel), layer 1 (channel x tap, taps
// past 5 zero), layer 3 (tap x channel, taps past 5 zero); plus the plain
// low-pass taps h[|i|] the net's output adds to.  w2, b1, b3 are contiguous.
struct __align__(16) NetWeights {
    uint16_t w2[kNetTaps * 256];
    uint16_t b1[256];
    uint16_t b3[256];
    float h[2 * kMaxTapD];
};

// Device side of the whole-volume host-buffer pipeline (slabs.cu).
struct HostPipe;
void free_host_pipe(HostPipe *hp);
// Buffers, streams and events of the slab-wise pipeline (slabs.cu), kept
// from one fdkod_reconstruct_slabs call to the next with the same slab size.
struct SlabPipe;
void free_slab_pipe(SlabPipe *sp);

struct PlanImpl {
    fdkod_geometry g{};
    int s = 0, D = 1, Pd = 1;
    fdkod_dtype qtype = FDKOD_F32;
    double2 *cs = nullptr;     // cos/sin of every view (host libm)
    SquareSet od;              // FDK-OD squares (level s)
    SquareSet pl;              // tiling used by the plain FDK baseline
    // filter stage
    int L = 0, log2L = 0;
    float *H = nullptr;        // ramp spectrum / L, real and even
    float2 *tw = nullptr;      // e^{-2 pi i m / L}, m < L
    float2 *tw2 = nullptr;     // L = 1024: e^{-2 pi i a b / 1024} at a * 32 + b, a, b < 32
    // angular low-pass of the decomposition (Sec. 2.1): symmetric taps
    // h[|i|], |i| < H D with H = tap_blocks (triangle by default, H = 1), and
    // per block offset r the weights of the 2H running sums,
    // tapw[r] = (w_0 .. w_{2H-1})
    int tap_blocks = 1;
    double htaps[2 * kMaxTapD] = {};
    float4 *tapw = nullptr;
    // learned decimation (null: the plain low-pass); net_host holds the
    // BF16-rounded weights as floats in the layout of the C interface
    NetWeights *net = nullptr;
    float net_host[kNetSize] = {};
    // decomposed data S'[q][j][v][t]
    float *Sp = nullptr;
    int Tstride = 0;
    int64_t sp_elems = 0;
    bool no_workspace = false; // made with FDKOD_PLAN_NO_WORKSPACE
    int *status = nullptr;     // device status word
    int64_t device_bytes = 0;
    // test hooks of the backprojection's failure paths (fdkod_set_test_fault)
    int test_fault = 0;
    int64_t wait_ns = 0;       // bounded-wait limit, 0 = the kernels' default
    // device buffers and streams of fdkod_reconstruct (made on its first call)
    HostPipe *pipe = nullptr;
    SlabPipe *slabs = nullptr;
};

// Raise a kernel's dynamic shared-memory limit only when a launch needs more
// than any earlier one on this device (one static record per kernel and
// device, the kernel being the template argument), so steady-state
// launches -- and launches recorded into a CUDA graph -- make no attribute
// call.
template <auto Kernel>
cudaError_t ensure_smem(size_t bytes) {
    constexpr int kDevices = 64;
    static std::atomic<size_t> set[kDevices];  // one record per kernel and device
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kDevices)
        return cudaFuncSetAttribute(Kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (bytes <= set[dev].load(std::memory_order_relaxed)) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(Kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) {
        size_t cur = set[dev].load();
        while (cur < bytes && !set[dev].compare_exchange_weak(cur, bytes)) {
        }
    }
    return e;
}

// host: backprojection staging windows of a square set (cs = cos/sin per view)
void size_windows(const PlanImpl &p, SquareSet &ss, const double2 *cs);

// host: angular low-pass taps h[|i|] (Sec. 2.1 leaves the kernel open):
// the triangle (D - |i|) / D^2, |i| < D, and a Hann-windowed sinc with its
// cutoff at the decimated Nyquist frequency, half-width H D, unit DC gain
void triangle_taps(int D, double *h);
void sinc_taps(int D, int H, double *h);
// host: running-sum weights per block offset r for taps of half-width H D:
// view j D + r adds w[r][m] = h[|r + (H - 1 - m) D|] (0 past the support) of
// its sample to decimated view j - H + 1 + m, m < 2H (H <= 2)
void tap_table(const double *h, int H, int D, float4 *w);

// Part of the volume and detector a launch works on: detector rows
// row0 .. row0 + nrows - 1 are the rows held by the source arrays (Q, the
// decomposed data), slices zoff .. zoff + nz - 1 are written to vol[z - zoff].
// The defaults (nrows, nz < 0) mean the whole detector and volume.
struct Band {
    int row0 = 0, nrows = -1, zoff = 0, nz = -1;
    // the filter and the decomposition only: the arrays hold the whole
    // detector ([P][Nv][...]) and the launch covers its rows row0 .. row0 +
    // nrows - 1 (instead of arrays that hold just those rows)
    bool whole_arrays = false;
};

// kernel launchers (return cudaError_t of the launch)
cudaError_t launch_bounds(const PlanImpl &p, SquareSet &ss, cudaStream_t st);
// views: how many views proj and Q hold (default: all P)
cudaError_t launch_filter(const PlanImpl &p, const float *proj, void *Q, cudaStream_t st, Band b = Band{},
                          int views = -1);
cudaError_t launch_decompose(const PlanImpl &p, const void *Q, float *out, cudaStream_t st, Band b = Band{});
cudaError_t launch_net_decompose(const PlanImpl &p, const void *Q, float *out, cudaStream_t st, int nrows);
// host: refresh the device copy of the net (weights from net_host, taps from htaps)
cudaError_t upload_net(PlanImpl &p);
cudaError_t launch_backproject(const PlanImpl &p, const SquareSet &ss, bool direct, const void *src,
                               float *vol, cudaStream_t st, Band b = Band{});
// The mirrored-pair backprojection of slice pairs p0 .. p1 - 1 (slices p and
// N - 1 - p, whole detector; vol is the whole volume); launched = false when
// the staged pair kernel does not apply (then nothing is launched).
cudaError_t launch_backproject_pairs(const PlanImpl &p, const SquareSet &ss, bool direct, const void *src,
                                     float *vol, cudaStream_t st, int p0, int p1, bool &launched);

// A batch of plans backprojected by one persistent launch (backproject.cu):
// per plan its FDK-OD source (Q when D = 1, else the decomposed data) and
// volume.  supported = false (and *out null) when a plan cannot take the
// persistent path (its windows are not float32 or do not fit a TMA box).
struct BatchImpl;
cudaError_t batch_create(const PlanImpl *const *plans, const void *const *src, float *const *vols, int count,
                         BatchImpl **out, bool &supported);
cudaError_t batch_launch(const BatchImpl &b, cudaStream_t st);
void batch_destroy(BatchImpl *b);

}  // namespace fdkod

struct fdkod_plan {
    fdkod::PlanImpl impl;
};
