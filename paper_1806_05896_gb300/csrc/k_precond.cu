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

// T: arithmetic (double, or float on the mixed path with FP32 copies of Theta)
template <typename T>
__global__ void k_zblock(GridDesc g, T a, const double* __restrict__ rw,
                         const double* __restrict__ rv, const T* __restrict__ thw,
                         const T* __restrict__ thv, double* __restrict__ zw,
                         double* __restrict__ zv) {
  int i, j, k;
  long long c;
  if (!interior_node(g, i, j, k, c)) return;
  T tw = thw[c], tv = thv[c];
  T det = a * (tw + tv) + tw * tv;  // (a + tw)(a + tv) - a^2
  T r1 = (T)rw[c], r2 = (T)rv[c];
  zw[c] = (double)(((a + tv) * r1 + a * r2) / det);
  zv[c] = (double)((a * r1 + (a + tw) * r2) / det);
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
    if (st.heat) {
      ly = st.heat_L(Ld<double>{zy}, c, -1);
    } else if (L.coef == nullptr) {
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

// ---------------------------------------------------------------------------
// Mixed-precision P_T pieces with float-float data (2D Poisson), at FP32 instruction
// rates: the z-block from FP32 right-hand sides, the Schur coupling and the
// (M + Theta_y) product in float-float arithmetic.
// ---------------------------------------------------------------------------
// Q1 mass action without the h^2/36 factor, float-float (rows [1 4 1] (x) [1 4 1])
template <typename LD>
IPM_D FF mass2_raw_ff(const LD& x, long long c, long long p) {
  auto row = [&](long long q) {
    const FF a = x(q - 1), b = x(q), d = x(q + 1);
    return ff_add(ff_add(a, FF{4.f * b.h, 4.f * b.l}), d);
  };
  const FF r1 = row(c);
  return ff_add(ff_add(row(c - p), FF{4.f * r1.h, 4.f * r1.l}), row(c + p));
}

// z_w, z_v from FP32 right-hand sides (FP64 results and FP32 copies)
__global__ void k_zblock32f(GridDesc g, float a, const float* __restrict__ rw,
                            const float* __restrict__ rv, const float* __restrict__ thw,
                            const float* __restrict__ thv, double* __restrict__ zw,
                            double* __restrict__ zv, float* __restrict__ zw32,
                            float* __restrict__ zv32) {
  int i, j, k;
  long long c;
  if (!interior_node(g, i, j, k, c)) return;
  const float tw = thw[c], tv = thv[c];
  const float det = a * (tw + tv) + tw * tv;
  const float r1 = rw[c], r2 = rv[c];
  const float w = ((a + tv) * r1 + a * r2) / det;
  const float v = (a * r1 + (a + tw) * r2) / det;
  zw[c] = (double)w;
  zv[c] = (double)v;
  zw32[c] = w;
  zv32[c] = v;
}

// t = L z_y - M (z_w - z_v) - r_p (z_* FP32, r_p and t float-float planes)
__global__ void k_coupling_ff(GridDesc g, FF mscale, FF third, const float* __restrict__ zy,
                              const float* __restrict__ zw, const float* __restrict__ zv,
                              const float* __restrict__ rph, const float* __restrict__ rpl,
                              float* __restrict__ th, float* __restrict__ tl) {
  int i, j, k;
  long long c;
  if (!interior_node(g, i, j, k, c)) return;
  const long long p = g.pitch;
  // L z_y = (8 z_c - sum of the 8 neighbours) / 3
  FF S = FF{zy[c - p - 1], 0.f};
  const long long nb[7] = {c - p, c - p + 1, c - 1, c + 1, c + p - 1, c + p, c + p + 1};
#pragma unroll
  for (int q = 0; q < 7; ++q) S = ff_add(S, FF{zy[nb[q]], 0.f});
  const FF Ly = ff_mul(ff_add(FF{8.f * zy[c], 0.f}, ff_neg(S)), third);
  auto dwv = [&](long long q) { return ff_two_sum(zw[q], -zv[q]); };
  const FF Ms = ff_mul(mass2_raw_ff(dwv, c, p), mscale);
  const FF t = ff_add(ff_add(Ly, ff_neg(Ms)), FF{-rph[c], -rpl[c]});
  th[c] = t.h;
  tl[c] = t.l;
}

// out = M s + Theta_y s (float-float planes; Theta_y as float-float planes)
__global__ void k_mass_theta_ff(GridDesc g, FF mscale, const float* __restrict__ sh,
                                const float* __restrict__ sl, const float* __restrict__ tyh,
                                const float* __restrict__ tyl, float* __restrict__ oh,
                                float* __restrict__ ol) {
  int i, j, k;
  long long c;
  if (!interior_node(g, i, j, k, c)) return;
  auto x = [&](long long q) { return FF{sh[q], sl[q]}; };
  const FF m = ff_mul(mass2_raw_ff(x, c, g.pitch), mscale);
  const FF r = ff_add(m, ff_mul(FF{tyh[c], tyl[c]}, x(c)));
  oh[c] = r.h;
  ol[c] = r.l;
}

template <typename Ti, typename To>
__global__ void k_convert(long long n, const Ti* __restrict__ x, To* __restrict__ y) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x)
    y[t] = (To)x[t];
}


// ---------------------------------------------------------------------------
// Partial observation: P_Pi (the subsection on partial observations)
// ---------------------------------------------------------------------------
// diagonals of the V-cycle operators of S_Pi_hat = (L^T + M_l) L^{-1} (L + M_r):
// m_l = row sums of M_s + Theta_y (the observed element masses lumped), and
// m_r = D zeta D, the lumped M_bar Z^{-1} M_bar^T with the z-block Z = alpha D~_M + Theta_z,
// zeta = (theta_w + theta_v) / (a (theta_w + theta_v) + theta_w theta_v), a = alpha D_M
__global__ void k_pi_diags(GridDesc g, double a, double d, const double* __restrict__ thy,
                           const double* __restrict__ thw, const double* __restrict__ thv,
                           double* __restrict__ ml, double* __restrict__ mr) {
  int i, j, k;
  long long c;
  if (!interior_node(g, i, j, k, c)) return;
  const long long p = g.pitch, pl = g.plane;
  const int ne = g.dim == 3 ? 8 : 4;
  int nobs = 0;
  for (int e = 0; e < ne; ++e) {
    const long long base = c - (e & 1) - ((e >> 1) & 1) * p - ((e >> 2) & 1) * pl;
    nobs += g.obs == nullptr || g.obs[base] != 0.f;
  }
  const double elem_row = g.dim == 3 ? g.h * g.h * g.h / 8.0 : g.h * g.h / 4.0;  // (h/2)^d
  ml[c] = nobs * elem_row + thy[c];
  const double tw = thw[c], tv = thv[c];
  mr[c] = d * d * (tw + tv) / (a * (tw + tv) + tw * tv);
}

// out = (M_s + Theta_y) x - r
__global__ void k_track_theta_minus(GridDesc g, Stencil<double> st, const double* __restrict__ x,
                                    const double* __restrict__ thy, const double* __restrict__ r,
                                    double* __restrict__ out) {
  int i, j, k;
  long long c;
  if (!interior_node(g, i, j, k, c)) return;
  out[c] = st.track(x, c) + thy[c] * x[c] - r[c];
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
  k_zblock<double><<<interior_grid(g), interior_block(), 0, s>>>(g, adM, rw, rv, thw, thv, zw, zv);
}
void launch_zblock32(const GridDesc& g, double adM, const double* rw, const double* rv,
                     const float* thw, const float* thv, double* zw, double* zv, cudaStream_t s) {
  count_launches(1);
  k_zblock<float><<<interior_grid(g), interior_block(), 0, s>>>(g, (float)adM, rw, rv, thw, thv, zw,
                                                               zv);
}
static FF ff_host(double x) {
  const float h = (float)x;
  return FF{h, (float)(x - (double)h)};
}
void launch_zblock32f(const GridDesc& g, double adM, const float* rw, const float* rv,
                      const float* thw, const float* thv, double* zw, double* zv, float* zw32,
                      float* zv32, cudaStream_t s) {
  count_launches(1);
  k_zblock32f<<<interior_grid(g), interior_block(), 0, s>>>(g, (float)adM, rw, rv, thw, thv, zw,
                                                            zv, zw32, zv32);
}
void launch_coupling_ff(const GridDesc& g, const float* zy, const float* zw, const float* zv,
                        const float* rph, const float* rpl, float* th, float* tl, cudaStream_t s) {
  count_launches(1);
  k_coupling_ff<<<interior_grid(g), interior_block(), 0, s>>>(
      g, ff_host(g.h * g.h / 36.0), ff_host(1.0 / 3.0), zy, zw, zv, rph, rpl, th, tl);
}
void launch_mass_theta_ff(const GridDesc& g, const float* sh, const float* sl, const float* tyh,
                          const float* tyl, float* oh, float* ol, cudaStream_t s) {
  count_launches(1);
  k_mass_theta_ff<<<interior_grid(g), interior_block(), 0, s>>>(g, ff_host(g.h * g.h / 36.0), sh,
                                                                sl, tyh, tyl, oh, ol);
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

void launch_pi_diags(const GridDesc& g, double a, double d, const double* thy, const double* thw,
                     const double* thv, double* ml, double* mr, cudaStream_t s) {
  count_launches(1);
  k_pi_diags<<<interior_grid(g), interior_block(), 0, s>>>(g, a, d, thy, thw, thv, ml, mr);
}

void launch_track_theta_minus(const GridDesc& g, const double* x, const double* thy,
                              const double* r, double* out, cudaStream_t s) {
  count_launches(1);
  k_track_theta_minus<<<interior_grid(g), interior_block(), 0, s>>>(g, make_stencil<double>(g), x,
                                                                      thy, r, out);
}
