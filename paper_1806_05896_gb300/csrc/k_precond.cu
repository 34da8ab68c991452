// Preconditioner kernels for P_D and P_T (Section 4).
//
// * (M + Theta_y)^{-1} by Chebyshev semi-iteration with the Jacobi splitting
//   D_M + Theta_y (Section 4.1; 20 steps in Section 5). The eigenvalues of
//   (D_M + Theta_y)^{-1}(M + Theta_y) lie in [min(l_min, 1), max(l_max, 1)] of
//   D_M^{-1} M, i.e. [1/4, 9/4] (2D Q1) and [1/8, 27/8] (3D Q1). The iteration
//   is written in its two-term form
//     x_{k+1} = x_k + (w_k - 1)(x_k - x_{k-1}) + (w_k / theta) J^{-1}(b - A x_k),
//   theta the interval centre, w_k from the Chebyshev three-term recurrence.
// * (alpha D~_M + Theta_z)^{-1}: independent 2x2 solves per node (Section 4.1).
// * The coupling row of P_T: t = L x_y - M x_w + M x_v - r_p (Section 4.2).
// * (M + Theta_y) s inside S_hat^{-1} (SchurApprox).
#include "kernels.h"

namespace {

template <typename T>
__global__ void k_cheb_init(GridDesc g, const double* __restrict__ b, const T* __restrict__ thy,
                            T dM, T inv_theta, T* __restrict__ bT, T* __restrict__ x1,
                            T* __restrict__ x0) {
  int i, j, k;
  long long c;
  if (!interior_node(g, i, j, k, c)) return;
  T bb = (T)b[c];
  bT[c] = bb;
  x1[c] = inv_theta * bb / (dM + thy[c]);
  x0[c] = T(0);
}

// out may alias xp (pointwise use only)
template <typename T, typename To>
__global__ void k_cheb_step(GridDesc g, Stencil<T> st, const T* __restrict__ xc, const T* xp,
                            const T* __restrict__ bT, const T* __restrict__ thy, T dM, T omega,
                            T inv_theta, To* out) {
  int i, j, k;
  long long c;
  if (!interior_node(g, i, j, k, c)) return;
  T x = xc[c];
  T th = thy[c];
  T ax = st.mass(xc, c) + th * x;
  T res = bT[c] - ax;
  T xn = x + (omega - T(1)) * (x - xp[c]) + omega * inv_theta * res / (dM + th);
  out[c] = (To)xn;
}

__global__ void k_zblock(GridDesc g, double a, const double* __restrict__ rw,
                         const double* __restrict__ rv, const double* __restrict__ thw,
                         const double* __restrict__ thv, double* __restrict__ zw,
                         double* __restrict__ zv) {
  int i, j, k;
  long long c;
  if (!interior_node(g, i, j, k, c)) return;
  double tw = thw[c], tv = thv[c];
  double det = a * (tw + tv) + tw * tv;  // (a + tw)(a + tv) - a^2
  double r1 = rw[c], r2 = rv[c];
  zw[c] = ((a + tv) * r1 + a * r2) / det;
  zv[c] = (a * r1 + (a + tw) * r2) / det;
}

template <typename T>
__global__ void k_coupling(GridDesc g, Stencil<double> st, OpL L, const double* __restrict__ zy,
                           const double* __restrict__ zw, const double* __restrict__ zv,
                           const double* __restrict__ rp, int triangular, T* __restrict__ t) {
  int i, j, k;
  long long c;
  if (!interior_node(g, i, j, k, c)) return;
  double v = -rp[c];
  if (triangular) {
    double ly;
    if (L.coef == nullptr) {
      ly = st.stiff(zy, c);
    } else {
      ly = 0.0;
#pragma unroll
      for (int o = 0; o < 9; ++o) {
        long long off = (long long)(o / 3 - 1) * st.p + (o % 3 - 1);
        ly += L.coef[o * g.field + c] * zy[c + off];
      }
    }
    v += ly - st.mass_f(LdDiff<double>{zw, zv}, c);
    t[c] = (T)v;
  } else {
    t[c] = (T)rp[c];
  }
}

template <typename T>
__global__ void k_mass_theta(GridDesc g, Stencil<T> st, const T* __restrict__ x,
                             const T* __restrict__ thy, T* __restrict__ out) {
  int i, j, k;
  long long c;
  if (!interior_node(g, i, j, k, c)) return;
  out[c] = st.mass(x, c) + thy[c] * x[c];
}

template <typename Ti, typename To>
__global__ void k_convert(long long n, const Ti* __restrict__ x, To* __restrict__ y) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x)
    y[t] = (To)x[t];
}

}  // namespace

template <typename T>
void launch_cheb_init(const GridDesc& g, const double* b, const T* thy, double dM, double inv_theta,
                      T* bT, T* x1, T* x0, cudaStream_t s) {
  count_launches(1);
  k_cheb_init<T><<<interior_grid(g), interior_block(), 0, s>>>(g, b, thy, (T)dM, (T)inv_theta, bT,
                                                               x1, x0);
}
template <typename T, typename To>
void launch_cheb_step(const GridDesc& g, const T* xc, const T* xp, const T* bT, const T* thy,
                      double dM, double omega, double inv_theta, To* out, cudaStream_t s) {
  count_launches(1);
  k_cheb_step<T, To><<<interior_grid(g), interior_block(), 0, s>>>(
      g, make_stencil<T>(g), xc, xp, bT, thy, (T)dM, (T)omega, (T)inv_theta, out);
}
void launch_zblock(const GridDesc& g, double adM, const double* rw, const double* rv,
                   const double* thw, const double* thv, double* zw, double* zv, cudaStream_t s) {
  count_launches(1);
  k_zblock<<<interior_grid(g), interior_block(), 0, s>>>(g, adM, rw, rv, thw, thv, zw, zv);
}
template <typename T>
void launch_coupling(const GridDesc& g, OpL L, const double* zy, const double* zw, const double* zv,
                     const double* rp, int triangular, T* t, cudaStream_t s) {
  count_launches(1);
  k_coupling<T><<<interior_grid(g), interior_block(), 0, s>>>(g, make_stencil<double>(g), L, zy, zw,
                                                              zv, rp, triangular, t);
}
template <typename T>
void launch_mass_theta(const GridDesc& g, const T* x, const T* thy, T* out, cudaStream_t s) {
  count_launches(1);
  k_mass_theta<T><<<interior_grid(g), interior_block(), 0, s>>>(g, make_stencil<T>(g), x, thy, out);
}
template <typename Ti, typename To>
void launch_convert(const GridDesc& g, const Ti* x, To* y, cudaStream_t s) {
  long long n = g.field;
  int blocks = (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
  count_launches(1);
  k_convert<Ti, To><<<blocks, 256, 0, s>>>(n, x, y);
}

template void launch_cheb_init<double>(const GridDesc&, const double*, const double*, double,
                                       double, double*, double*, double*, cudaStream_t);
template void launch_cheb_init<float>(const GridDesc&, const double*, const float*, double, double,
                                      float*, float*, float*, cudaStream_t);
template void launch_cheb_step<double, double>(const GridDesc&, const double*, const double*,
                                               const double*, const double*, double, double, double,
                                               double*, cudaStream_t);
template void launch_cheb_step<float, float>(const GridDesc&, const float*, const float*,
                                             const float*, const float*, double, double, double,
                                             float*, cudaStream_t);
template void launch_cheb_step<float, double>(const GridDesc&, const float*, const float*,
                                              const float*, const float*, double, double, double,
                                              double*, cudaStream_t);
template void launch_coupling<double>(const GridDesc&, OpL, const double*, const double*,
                                      const double*, const double*, int, double*, cudaStream_t);
template void launch_coupling<float>(const GridDesc&, OpL, const double*, const double*,
                                     const double*, const double*, int, float*, cudaStream_t);
template void launch_mass_theta<double>(const GridDesc&, const double*, const double*, double*,
                                        cudaStream_t);
template void launch_mass_theta<float>(const GridDesc&, const float*, const float*, float*,
                                       cudaStream_t);
template void launch_convert<double, float>(const GridDesc&, const double*, float*, cudaStream_t);
template void launch_convert<float, double>(const GridDesc&, const float*, double*, cudaStream_t);
template void launch_convert<double, double>(const GridDesc&, const double*, double*, cudaStream_t);
