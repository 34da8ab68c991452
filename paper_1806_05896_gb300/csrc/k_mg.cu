// Geometric multigrid kernels for A = L + diag(m) (the matrix L + M_hat of
// Section 4.2 and its coarse-grid counterparts).
//
// Hierarchy: grids of 2^k + 1 nodes per direction, coarse node I <-> fine node
// 2I. Transfer: P = bilinear (trilinear) interpolation, restriction P^T (full
// weighting, weights [1/2 1 1/2] per direction, unnormalised). Coarse
// operators: the Q1 stiffness rediscretised on the coarse grid (equal to
// P^T L P for nested Q1 spaces) plus the row-sum lumping of P^T diag(m) P,
// i.e. m_c = P^T m. Smoother: damped Jacobi with jinv = omega / diag(A).
// Transposed cycles (for L^T + M_hat) use L^T in every stencil.
#include "kernels.h"

namespace {

template <typename T>
IPM_D T op_apply(const OpL& L, const Stencil<T>& st, const T* __restrict__ x, long long c,
                 long long field, int transpose) {
  if (L.coef == nullptr) return st.stiff(x, c);
  const float* cf = L.coef32;
  const double* cd = L.coef;
  T acc = T(0);
#pragma unroll
  for (int o = 0; o < 9; ++o) {
    long long off = (long long)(o / 3 - 1) * st.p + (o % 3 - 1);
    long long idx = transpose ? (long long)(8 - o) * field + c + off : (long long)o * field + c;
    T cv = (sizeof(T) == 4 && cf) ? (T)cf[idx] : (T)cd[idx];
    acc += cv * x[c + off];
  }
  return acc;
}

template <typename T>
IPM_D T op_diag(const OpL& L, const GridDesc& g, long long c) {
  if (L.coef == nullptr) return g.dim == 2 ? T(8.0 / 3.0) : T(8.0 * g.h / 3.0);
  return (T)L.coef[4 * g.field + c];
}

template <typename T>
__global__ void k_mg_smooth(GridDesc g, Stencil<T> st, OpL L, const T* __restrict__ xin,
                            T* __restrict__ xout, const T* __restrict__ b, const T* __restrict__ m,
                            const T* __restrict__ jinv, int zero_init, int transpose) {
  int i, j, k;
  long long c;
  if (!interior_node(g, i, j, k, c)) return;
  if (zero_init) {
    xout[c] = jinv[c] * b[c];
    return;
  }
  T x = xin[c];
  T ax = op_apply<T>(L, st, xin, c, g.field, transpose) + m[c] * x;
  xout[c] = x + jinv[c] * (b[c] - ax);
}

template <typename T>
__global__ void k_mg_residual(GridDesc g, Stencil<T> st, OpL L, const T* __restrict__ x,
                              const T* __restrict__ b, const T* __restrict__ m, T* __restrict__ r,
                              int transpose) {
  int i, j, k;
  long long c;
  if (!interior_node(g, i, j, k, c)) return;
  r[c] = b[c] - (op_apply<T>(L, st, x, c, g.field, transpose) + m[c] * x[c]);
}

// b_c(I) = sum_{a in {-1,0,1}^d} prod_k w(a_k) r_f(2I + a),  w(0) = 1, w(+-1) = 1/2
template <typename T>
__global__ void k_mg_restrict(GridDesc gf, GridDesc gc, const T* __restrict__ rf,
                              T* __restrict__ bc) {
  int I, J, K;
  long long cc;
  if (!interior_node(gc, I, J, K, cc)) return;
  long long cf = node_index(gf, 2 * I, 2 * J, gf.dim == 3 ? 2 * K : 0);
  int p = gf.pitch;
  auto plane = [&](long long q) {
    T r0 = T(0.5) * rf[q - p - 1] + rf[q - p] + T(0.5) * rf[q - p + 1];
    T r1 = T(0.5) * rf[q - 1] + rf[q] + T(0.5) * rf[q + 1];
    T r2 = T(0.5) * rf[q + p - 1] + rf[q + p] + T(0.5) * rf[q + p + 1];
    return T(0.5) * r0 + r1 + T(0.5) * r2;
  };
  T v;
  if (gf.dim == 2) v = plane(cf);
  else v = T(0.5) * plane(cf - gf.plane) + plane(cf) + T(0.5) * plane(cf + gf.plane);
  bc[cc] = v;
}

// x_f(i) += (P x_c)(i): product over directions of the 1D linear interpolation
template <typename T>
__global__ void k_mg_prolong_add(GridDesc gf, GridDesc gc, const T* __restrict__ xc,
                                 T* __restrict__ xf) {
  int i, j, k;
  long long c;
  if (!interior_node(gf, i, j, k, c)) return;
  int i0 = i >> 1, j0 = j >> 1, k0 = k >> 1;
  int ni = (i & 1) ? 2 : 1, nj = (j & 1) ? 2 : 1, nk = (gf.dim == 3 && (k & 1)) ? 2 : 1;
  T wi = ni == 2 ? T(0.5) : T(1), wj = nj == 2 ? T(0.5) : T(1), wk = nk == 2 ? T(0.5) : T(1);
  T acc = T(0);
  for (int dk = 0; dk < nk; ++dk)
    for (int dj = 0; dj < nj; ++dj)
      for (int di = 0; di < ni; ++di)
        acc += xc[node_index(gc, i0 + di, j0 + dj, gf.dim == 3 ? k0 + dk : 0)];
  xf[c] += wi * wj * wk * acc;
}

template <typename T>
__global__ void k_mg_coarsest(GridDesc g, OpL L, const T* __restrict__ b, const T* __restrict__ m,
                              T* __restrict__ x) {
  // grid of 3 nodes per direction: one unknown at (1,1[,1])
  long long c = node_index(g, 1, 1, g.dim == 3 ? 1 : 0);
  x[c] = b[c] / (op_diag<T>(L, g, c) + m[c]);
}

template <typename T>
__global__ void k_mg_jinv(GridDesc g, OpL L, const T* __restrict__ m, T omega, T* __restrict__ jinv) {
  int i, j, k;
  long long c;
  if (!interior_node(g, i, j, k, c)) return;
  jinv[c] = omega / (op_diag<T>(L, g, c) + m[c]);
}

template <typename T>
__global__ void k_mg_zero(GridDesc g, T* __restrict__ x) {
  int i, j, k;
  long long c;
  if (!interior_node(g, i, j, k, c)) return;
  x[c] = T(0);
}

// Outer step of the mixed-precision multigrid solve on the finest level:
// x_new = x_prev + e (x_prev may be null = 0) in FP64, and, if r32 is given,
// r32 = b - (L + diag(m)) x_new in FP64 rounded to FP32 (the next FP32 cycle's
// right-hand side). The stencil reads x_prev + e at the neighbours directly.
__global__ void k_mg_outer(GridDesc g, Stencil<double> st, OpL L, const double* __restrict__ xprev,
                           const float* __restrict__ e, const double* __restrict__ b,
                           const double* __restrict__ m, double* __restrict__ xnew,
                           float* __restrict__ r32, int transpose) {
  int i, j, k;
  long long c;
  if (!interior_node(g, i, j, k, c)) return;
  struct Sum {
    const double* a;
    const float* e;
    IPM_D double operator()(long long q) const { return (a ? a[q] : 0.0) + (double)e[q]; }
  } xn{xprev, e};
  double x = xn(c);
  xnew[c] = x;
  if (r32) {
    double ax;
    if (L.coef == nullptr) {
      ax = st.stiff_f(xn, c);
    } else {
      ax = 0.0;
#pragma unroll
      for (int o = 0; o < 9; ++o) {
        long long off = (long long)(o / 3 - 1) * st.p + (o % 3 - 1);
        long long idx = transpose ? (long long)(8 - o) * g.field + c + off : (long long)o * g.field + c;
        ax += L.coef[idx] * xn(c + off);
      }
    }
    r32[c] = (float)(b[c] - (ax + m[c] * x));
  }
}

// ---------------------------------------------------------------------------
// Outer residual of the mixed multigrid solve in float-float arithmetic (2D Poisson).
// Float-float arithmetic (FF, common.cuh): the residual's absolute error is ~1e-13 |x|,
// far below what the FP32 cycles resolve, at FP32 instruction rates.
// ---------------------------------------------------------------------------
// x' = x + e (x = 0 when `first`), and either out64 = x' (last cycle) or
// x' -> (xh_out, xl_out) and r32 = b - (L + diag m) x' rounded to FP32, evaluated as
// (3b - (8 x'_c - sum of the 8 neighbours) - 3m x'_c) / 3. `first` also stores 3b
// (from b64) as float-float for the later cycles; m3 = 3m as float-float.
// The right-hand side comes as FP64 (b64) or as float-float planes (bff: high parts, then
// low parts, g.field apart); the last cycle's x' goes to out64 or to float-float planes.
__global__ void k_mg_outer_ff(GridDesc g, const float* __restrict__ xh_in,
                              const float* __restrict__ xl_in, const float* __restrict__ e,
                              const double* __restrict__ b64, const float* __restrict__ bff,
                              float* __restrict__ b3h, float* __restrict__ b3l,
                              const float* __restrict__ m3h, const float* __restrict__ m3l,
                              float* __restrict__ xh_out, float* __restrict__ xl_out,
                              float* __restrict__ r32, double* __restrict__ out64,
                              float* __restrict__ outff, int first) {
  int i, j, k;
  long long c;
  if (!interior_node(g, i, j, k, c)) return;
  auto xq = [&](long long q) -> FF {
    if (first) return {e[q], 0.f};
    const FF s = ff_two_sum(xh_in[q], e[q]);
    return ff_fast_two_sum(s.h, __fadd_rn(s.l, xl_in[q]));
  };
  const FF xc = xq(c);
  if (out64) {
    out64[c] = (double)xc.h + (double)xc.l;
    return;
  }
  if (outff) {
    outff[c] = xc.h;
    outff[g.field + c] = xc.l;
    return;
  }
  xh_out[c] = xc.h;
  xl_out[c] = xc.l;
  FF b3;
  if (first) {
    b3 = bff ? ff_mul(FF{bff[c], bff[g.field + c]}, FF{3.f, 0.f}) : ff_from_double(3.0 * b64[c]);
    b3h[c] = b3.h;
    b3l[c] = b3.l;
  } else {
    b3 = {b3h[c], b3l[c]};
  }
  const long long p = g.pitch;
  FF S = xq(c - p - 1);
  S = ff_add(S, xq(c - p));
  S = ff_add(S, xq(c - p + 1));
  S = ff_add(S, xq(c - 1));
  S = ff_add(S, xq(c + 1));
  S = ff_add(S, xq(c + p - 1));
  S = ff_add(S, xq(c + p));
  S = ff_add(S, xq(c + p + 1));
  const FF d = ff_add({8.f * xc.h, 8.f * xc.l}, ff_neg(S));
  const FF mx = ff_mul({m3h[c], m3l[c]}, xc);
  const FF R = ff_add(b3, ff_neg(ff_add(d, mx)));
  r32[c] = __fdiv_rn(__fadd_rn(R.h, R.l), 3.0f);
}

// (hi, lo) = 3 m as float-float
__global__ void k_split3_ff(GridDesc g, const double* __restrict__ m, float* __restrict__ hi,
                            float* __restrict__ lo) {
  int i, j, k;
  long long c;
  if (!interior_node(g, i, j, k, c)) return;
  const FF v = ff_from_double(3.0 * m[c]);
  hi[c] = v.h;
  lo[c] = v.l;
}

}  // namespace

void launch_mg_outer(const GridDesc& g, OpL L, const double* xprev, const float* e,
                     const double* b, const double* m, double* xnew, float* r32, int transpose,
                     cudaStream_t s) {
  count_launches(1);
  k_mg_outer<<<interior_grid(g), interior_block(), 0, s>>>(g, make_stencil<double>(g), L, xprev, e,
                                                           b, m, xnew, r32, transpose);
}

void launch_mg_outer_ff(const GridDesc& g, const float* xh_in, const float* xl_in, const float* e,
                        const double* b64, const float* bff, float* b3h, float* b3l,
                        const float* m3h, const float* m3l, float* xh_out, float* xl_out,
                        float* r32, double* out64, float* outff, int first, cudaStream_t s) {
  count_launches(1);
  k_mg_outer_ff<<<interior_grid(g), interior_block(), 0, s>>>(g, xh_in, xl_in, e, b64, bff, b3h,
                                                              b3l, m3h, m3l, xh_out, xl_out, r32,
                                                              out64, outff, first);
}

void launch_split3_ff(const GridDesc& g, const double* m, float* hi, float* lo, cudaStream_t s) {
  count_launches(1);
  k_split3_ff<<<interior_grid(g), interior_block(), 0, s>>>(g, m, hi, lo);
}

template <typename T>
void launch_mg_smooth(const GridDesc& g, OpL L, const T* xin, T* xout, const T* b, const T* m,
                      const T* jinv, int zero_init, int transpose, cudaStream_t s) {
  count_launches(1);
  k_mg_smooth<T><<<interior_grid(g), interior_block(), 0, s>>>(g, make_stencil<T>(g), L, xin, xout,
                                                               b, m, jinv, zero_init, transpose);
}
template <typename T>
void launch_mg_residual(const GridDesc& g, OpL L, const T* x, const T* b, const T* m, T* r,
                        int transpose, cudaStream_t s) {
  count_launches(1);
  k_mg_residual<T><<<interior_grid(g), interior_block(), 0, s>>>(g, make_stencil<T>(g), L, x, b, m,
                                                                 r, transpose);
}
template <typename T>
void launch_mg_restrict(const GridDesc& gf, const GridDesc& gc, const T* rf, T* bc, cudaStream_t s) {
  count_launches(1);
  k_mg_restrict<T><<<interior_grid(gc), interior_block(), 0, s>>>(gf, gc, rf, bc);
}
template <typename T>
void launch_mg_prolong_add(const GridDesc& gf, const GridDesc& gc, const T* xc, T* xf,
                           cudaStream_t s) {
  count_launches(1);
  k_mg_prolong_add<T><<<interior_grid(gf), interior_block(), 0, s>>>(gf, gc, xc, xf);
}
template <typename T>
void launch_mg_coarsest(const GridDesc& g, OpL L, const T* b, const T* m, T* x, cudaStream_t s) {
  count_launches(1);
  k_mg_coarsest<T><<<1, 1, 0, s>>>(g, L, b, m, x);
}
template <typename T>
void launch_mg_jinv(const GridDesc& g, OpL L, const T* m, double omega, T* jinv, cudaStream_t s) {
  count_launches(1);
  k_mg_jinv<T><<<interior_grid(g), interior_block(), 0, s>>>(g, L, m, (T)omega, jinv);
}
template <typename T>
void launch_mg_zero(const GridDesc& g, T* x, cudaStream_t s) {
  count_launches(1);
  k_mg_zero<T><<<interior_grid(g), interior_block(), 0, s>>>(g, x);
}

#define IPM_MG_INST(T)                                                                          \
  template void launch_mg_smooth<T>(const GridDesc&, OpL, const T*, T*, const T*, const T*,      \
                                    const T*, int, int, cudaStream_t);                           \
  template void launch_mg_residual<T>(const GridDesc&, OpL, const T*, const T*, const T*, T*, int, \
                                      cudaStream_t);                                              \
  template void launch_mg_restrict<T>(const GridDesc&, const GridDesc&, const T*, T*, cudaStream_t); \
  template void launch_mg_prolong_add<T>(const GridDesc&, const GridDesc&, const T*, T*,          \
                                         cudaStream_t);                                           \
  template void launch_mg_coarsest<T>(const GridDesc&, OpL, const T*, const T*, T*, cudaStream_t); \
  template void launch_mg_jinv<T>(const GridDesc&, OpL, const T*, double, T*, cudaStream_t);     \
  template void launch_mg_zero<T>(const GridDesc&, T*, cudaStream_t);
IPM_MG_INST(float)
IPM_MG_INST(double)
