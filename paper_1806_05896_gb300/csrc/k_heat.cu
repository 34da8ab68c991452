// All-at-once heat equation (Section 3.4): the time-level sweeps of the Schur-complement
// approximation (calL + M_hat)(tau calM + Theta_y)^{-1}(calL + M_hat)^T.
//
// With backward Euler in time, calL is block lower bidiagonal: (M + tau K) on the
// diagonal and -M below it. A solve with calL + M_hat therefore runs forward over the time
// levels, each level a 2D solve with M + tau K + diag(M_hat_k) for the right-hand side
// t_k + M x_{k-1}; its transpose runs backward with t_k + M x_{k+1}. The 2D solves are
// FP32 V-cycles of the one-CTA coarse kernel (k_mg_fused.cu) on each level's own
// hierarchy; the kernels here form each level's right-hand side in FP64 and carry the
// FP32 results back to FP64.
#include "kernels.h"

namespace {

// b32 = (float)(t_k + M x_prev) on the interior of plane k, where x_prev is plane kp of
// the FP32 results (kp < 0: no previous level); the FP64 copy of plane kp is written to x64.
__global__ void k_heat_plane_rhs(GridDesc g, const double* __restrict__ t, int k, int kp,
                                 const float* __restrict__ x32, double* __restrict__ x64,
                                 float* __restrict__ b32) {
  const int i = 1 + blockIdx.x * blockDim.x + threadIdx.x;
  const int j = 1 + blockIdx.y * blockDim.y + threadIdx.y;
  if (i > g.n - 2 || j > g.n - 2) return;
  const long long p = g.pitch;
  const long long c = (long long)k * g.plane + (long long)j * p + i;
  double v = t[c];
  if (kp >= 0) {
    const long long q = (long long)kp * g.plane + (long long)j * p + i;
    auto ld = [&](long long a) { return (double)x32[a]; };
    const double s = (ld(q - p - 1) + 4.0 * ld(q - p) + ld(q - p + 1)) +
                     4.0 * (ld(q - 1) + 4.0 * ld(q) + ld(q + 1)) +
                     (ld(q + p - 1) + 4.0 * ld(q + p) + ld(q + p + 1));
    v += (g.h * g.h / 36.0) * s;
    x64[q] = ld(q);
  }
  b32[c] = (float)v;
}

__global__ void k_heat_plane_store(GridDesc g, int k, const float* __restrict__ x32,
                                   double* __restrict__ x64) {
  const int i = 1 + blockIdx.x * blockDim.x + threadIdx.x;
  const int j = 1 + blockIdx.y * blockDim.y + threadIdx.y;
  if (i > g.n - 2 || j > g.n - 2) return;
  const long long c = (long long)k * g.plane + (long long)j * g.pitch + i;
  x64[c] = (double)x32[c];
}

dim3 plane_grid(const GridDesc& g) {
  const int m = g.n - 2;
  return dim3((m + 31) / 32, (m + 7) / 8, 1);
}

}  // namespace

void launch_heat_plane_rhs(const GridDesc& g, const double* t, int k, int kp, const float* x32,
                           double* x64, float* b32, cudaStream_t s) {
  count_launches(1);
  k_heat_plane_rhs<<<plane_grid(g), dim3(32, 8, 1), 0, s>>>(g, t, k, kp, x32, x64, b32);
}

void launch_heat_plane_store(const GridDesc& g, int k, const float* x32, double* x64,
                             cudaStream_t s) {
  count_launches(1);
  k_heat_plane_store<<<plane_grid(g), dim3(32, 8, 1), 0, s>>>(g, k, x32, x64);
}
