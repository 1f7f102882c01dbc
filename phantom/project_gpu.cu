// Seeded-input generator on the GPU: closed-form ellipsoid line integrals
// for workloads too large for the CPU generator (project.c).  Input
// generation only -- no reconstruction arithmetic; the oracle never reads
// its output.  Same geometry and ellipsoid parameter block as project.c.
//
// For a ray from source S through detector point T (virtual detector at the
// isocentre), an ellipsoid with centre c, rotation Q and semi-axes (A,B,C)
// maps to the unit sphere by M = diag(1/A,1/B,1/C) Q^T.  With t' = M (T - c)
// (a small, well-conditioned vector) and the unit direction
// e = M (T - S) / |M (T - S)|, the ray's closest approach to the sphere
// centre is m = t' - (t'.e) e, and the chord is
// 2 sqrt(1 - |m|^2) |T - S| / |M (T - S)| when |m| < 1.  FP32 throughout.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

namespace {

constexpr int kMaxEll = 512;
__constant__ float c_ell[kMaxEll * 16];

__global__ void project_kernel(int n_ell, float R, int Nu, int Nv, int P, int k0, float *__restrict__ out) {
    const int u = blockIdx.x * blockDim.x + threadIdx.x;
    const int v = blockIdx.y * blockDim.y + threadIdx.y;
    const int kk = blockIdx.z;
    if (u >= Nu || v >= Nv) return;
    const int k = k0 + kk;
    const double beta = 2.0 * M_PI * (double)k / (double)P;
    const float cb = (float)cos(beta), sb = (float)sin(beta);
    const float a = (float)u - 0.5f * (float)(Nu - 1);
    const float b = (float)v - 0.5f * (float)(Nv - 1);
    const float T[3] = {-a * sb, a * cb, b};
    const float d[3] = {T[0] + R * cb, T[1] + R * sb, T[2]};  // T - S
    const float dlen = sqrtf(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    float acc = 0.f;
    for (int e = 0; e < n_ell; ++e) {
        const float *E = c_ell + 16 * e;
        const float tc[3] = {T[0] - E[0], T[1] - E[1], T[2] - E[2]};
        float tp[3], dp[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            // column i of Q is body axis i: (Q^T x)_i = sum_r Q[r][i] x_r
            tp[i] = (E[6 + i] * tc[0] + E[9 + i] * tc[1] + E[12 + i] * tc[2]) / E[3 + i];
            dp[i] = (E[6 + i] * d[0] + E[9 + i] * d[1] + E[12 + i] * d[2]) / E[3 + i];
        }
        const float dn = sqrtf(dp[0] * dp[0] + dp[1] * dp[1] + dp[2] * dp[2]);
        const float inv = 1.0f / dn;
        const float ex = dp[0] * inv, ey = dp[1] * inv, ez = dp[2] * inv;
        const float te = tp[0] * ex + tp[1] * ey + tp[2] * ez;
        const float mx = tp[0] - te * ex, my = tp[1] - te * ey, mz = tp[2] - te * ez;
        const float m2 = mx * mx + my * my + mz * mz;
        if (m2 < 1.0f) acc += E[15] * 2.0f * sqrtf(1.0f - m2) * dlen * inv;
    }
    out[((size_t)kk * Nv + v) * Nu + u] = acc;
}

}  // namespace

// Views k0 .. k1-1 into out (device, [k1-k0][Nv][Nu] float32), enqueued on
// `stream`.  ell: host [n_ell][16] float32 (the block layout of project.c).
// Returns 0, -1 for bad arguments, -2 for a CUDA error.
extern "C" int phantom_project_gpu(int n_ell, const float *ell, double R, int Nu, int Nv, int P, int k0, int k1,
                                   float *out, uintptr_t stream) {
    if (n_ell < 0 || n_ell > kMaxEll || Nu <= 0 || Nv <= 0 || P <= 0 || k0 < 0 || k1 > P || k0 >= k1 || !out)
        return -1;
    cudaStream_t st = (cudaStream_t)stream;
    if (n_ell > 0 &&
        cudaMemcpyToSymbolAsync(c_ell, ell, sizeof(float) * 16 * (size_t)n_ell, 0, cudaMemcpyHostToDevice, st) !=
            cudaSuccess)
        return -2;
    dim3 block(32, 8);
    dim3 grid((Nu + 31) / 32, (Nv + 7) / 8, k1 - k0);
    project_kernel<<<grid, block, 0, st>>>(n_ell, (float)R, Nu, Nv, P, k0, out);
    if (cudaGetLastError() != cudaSuccess) return -2;
    return cudaStreamSynchronize(st) == cudaSuccess ? 0 : -2;
}
