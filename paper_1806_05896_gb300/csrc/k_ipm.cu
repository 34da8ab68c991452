// Interior point kernels: data set-up, barrier diagonals and Newton right-hand
// side, step lengths, iterate update, feasibility/complementarity measures, and
// the matrix-free saddle-point operator of the reduced Newton system.
//
// Pearson, Porcelli, Stoll (2018): Section 3 (NewtonSystem), (zupdate1-4),
// (prdu), (gap); Section 4.2 (the diagonal M_hat); Appendix Algorithm A.1.
#include "kernels.h"
#include <cmath>

namespace {

// ---------------------------------------------------------------------------
// Elliptic operator L and its transpose at an interior node.
// ---------------------------------------------------------------------------
template <typename T, typename F>
IPM_D T apply_L(const OpL& L, const Stencil<T>& st, const F& f, long long c, long long field) {
  if (st.heat) return st.heat_L(f, c, -1);
  if (L.coef == nullptr) return st.stiff_f(f, c);
  T acc = T(0);
#pragma unroll
  for (int o = 0; o < 9; ++o) {
    long long off = (long long)(o / 3 - 1) * st.p + (o % 3 - 1);
    acc += (T)L.coef[o * field + c] * f(c + off);
  }
  return acc;
}
// (L^T x)_i = sum_q L[i + off_q, i] x_{i + off_q} = sum_q coef[opp(q)][i + off_q] x_{i + off_q};
// coefficients are zero at non-interior nodes.
template <typename T, typename F>
IPM_D T apply_LT(const OpL& L, const Stencil<T>& st, const F& f, long long c, long long field) {
  if (st.heat) return st.heat_L(f, c, +1);
  if (L.coef == nullptr) return st.stiff_f(f, c);
  T acc = T(0);
#pragma unroll
  for (int o = 0; o < 9; ++o) {
    long long off = (long long)(o / 3 - 1) * st.p + (o % 3 - 1);
    acc += (T)L.coef[(8 - o) * field + c + off] * f(c + off);
  }
  return acc;
}

struct Inv {  // reciprocal distances to present bounds, zero for absent ones
  double ya, yb, wa, wb, va, vb;
  bool hya, hyb, hwb, hvb;
};

IPM_D Inv inv_dist(const IpmBounds& b, double y, double w, double v, long long c) {
  Inv r;
  double ya = b.ya[c], yb = b.yb[c], zbw = b.zbw[c], zbv = b.zbv[c];
  r.hya = isfinite(ya);
  r.hyb = isfinite(yb);
  r.hwb = isfinite(zbw);
  r.hvb = isfinite(zbv);
  r.ya = r.hya ? 1.0 / (y - ya) : 0.0;
  r.yb = r.hyb ? 1.0 / (yb - y) : 0.0;
  r.wa = 1.0 / w;  // z_a = 0: the lower bounds of w and v always exist
  r.wb = r.hwb ? 1.0 / (zbw - w) : 0.0;
  r.va = 1.0 / v;
  r.vb = r.hvb ? 1.0 / (zbv - v) : 0.0;
  return r;
}

// ---------------------------------------------------------------------------
__global__ void k_pack(GridDesc g, const double* __restrict__ dense, double* __restrict__ out,
                       int mode) {
  long long nn = (long long)g.n * g.n * (g.dim == 3 ? g.n : 1);
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nn;
       t += (long long)gridDim.x * blockDim.x) {
    int i = (int)(t % g.n);
    int j = (int)((t / g.n) % g.n);
    int k = g.dim == 3 ? (int)(t / ((long long)g.n * g.n)) : 0;
    bool bnd = i == 0 || j == 0 || i == g.n - 1 || j == g.n - 1 ||
               (g.dim == 3 && (k == 0 || k == g.n - 1));
    double v = dense ? dense[t] : 0.0;
    if (mode == 1 && bnd) v = 0.0;   // interior only
    if (mode == 2 && !bnd) v = 0.0;  // boundary only (Dirichlet lift)
    out[node_index(g, i, j, k)] = v;
  }
}

__global__ void k_unpack(GridDesc g, const double* __restrict__ in, const double* __restrict__ bnd,
                         double* __restrict__ dense) {
  long long nn = (long long)g.n * g.n * (g.dim == 3 ? g.n : 1);
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nn;
       t += (long long)gridDim.x * blockDim.x) {
    int i = (int)(t % g.n);
    int j = (int)((t / g.n) % g.n);
    int k = g.dim == 3 ? (int)(t / ((long long)g.n * g.n)) : 0;
    bool isb = i == 0 || j == 0 || i == g.n - 1 || j == g.n - 1 ||
               (g.dim == 3 && (k == 0 || k == g.n - 1));
    long long c = node_index(g, i, j, k);
    dense[t] = isb ? (bnd ? bnd[c] : 0.0) : in[c];
  }
}

// c_y = (M (y_d - g_lift))_I,  f = (M f)_I - (L g_lift)_I
__global__ void k_setup_data(GridDesc g, Stencil<double> st, const double* __restrict__ yd,
                             const double* __restrict__ f, const double* __restrict__ gl, OpL L,
                             double* __restrict__ cy, double* __restrict__ fv) {
  int i, j, k;
  long long c;
  if (!interior_node(g, i, j, k, c)) return;
  cy[c] = st.track_f(LdDiff<double>{yd, gl}, c);
  fv[c] = st.mass(f, c) - apply_L<double>(L, st, Ld<double>{gl}, c, g.field);
}

// sum over elements of r_e^T M_e r_e, r = y_d - g_lift, M_e = (h/6)^d (M1e (x) ... ), M1e = [2 1; 1 2]
__global__ void k_element_mass_form(GridDesc g, const double* __restrict__ yd,
                                    const double* __restrict__ gl, double* __restrict__ part) {
  __shared__ double sh[32];
  // heat layout: the 2D elements of every time level 1 .. n-2, weighted by tau
  const int edim = g.heat ? 2 : g.dim;
  long long ne1 = g.n - 1;
  long long ne = g.heat ? ne1 * ne1 * (g.n - 2) : (g.dim == 3 ? ne1 * ne1 * ne1 : ne1 * ne1);
  int nl = edim == 3 ? 8 : 4;
  double acc = 0.0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < ne;
       e += (long long)gridDim.x * blockDim.x) {
    int ex = (int)(e % ne1), ey = (int)((e / ne1) % ne1);
    int ez = g.dim == 3 ? (int)(e / (ne1 * ne1)) + (g.heat ? 1 : 0) : 0;
    if (g.obs && g.obs[node_index(g, ex, ey, ez)] == 0.f) continue;  // unobserved element
    double r[8];
    for (int l = 0; l < nl; ++l) {
      long long c = node_index(g, ex + (l & 1), ey + ((l >> 1) & 1), ez + ((l >> 2) & 1));
      r[l] = yd[c] - gl[c];
    }
    double q = 0.0;
    for (int a = 0; a < nl; ++a)
      for (int bb = 0; bb < nl; ++bb) {
        double wgt = 1.0;
        for (int kk = 0; kk < edim; ++kk) wgt *= (((a >> kk) & 1) == ((bb >> kk) & 1)) ? 2.0 : 1.0;
        q += wgt * r[a] * r[bb];
      }
    acc += q;
  }
  double s6 = g.h / 6.0;
  double scale = g.heat ? g.tau * s6 * s6 : (g.dim == 3 ? s6 * s6 * s6 : s6 * s6);
  double t = block_sum(acc * scale, sh);
  if (lin_tid() == 0) part[lin_block()] = t;
}

// ||c_y||^2, ||f||^2 and the number of present bounds
__global__ void k_setup_norms(GridDesc g, const double* __restrict__ cy,
                              const double* __restrict__ fv, IpmBounds b, double* __restrict__ part) {
  __shared__ double sh[32];
  int i, j, k;
  long long c;
  bool in = interior_node(g, i, j, k, c);
  double a0 = 0, a1 = 0, a2 = 0;
  if (in) {
    a0 = cy[c] * cy[c];
    a1 = fv[c] * fv[c];
    a2 = 2.0 + (isfinite(b.ya[c]) ? 1 : 0) + (isfinite(b.yb[c]) ? 1 : 0) +
         (isfinite(b.zbw[c]) ? 1 : 0) + (isfinite(b.zbv[c]) ? 1 : 0);
  }
  long long bi = lin_block();
  double t0 = block_sum(a0, sh), t1 = block_sum(a1, sh), t2 = block_sum(a2, sh);
  if (lin_tid() == 0) {
    part[bi * 3 + 0] = t0;
    part[bi * 3 + 1] = t1;
    part[bi * 3 + 2] = t2;
  }
}

// Central-path start: y^0 = 0 (or box centre / unit offset), z^0 = (z_a + z_b)/2
// (z_a + 1 if z_b absent), p^0 = 0, lambda^0 = mu^0 / distance.
__global__ void k_init_state(GridDesc g, IpmBounds b, IpmState s, double mu0) {
  int i, j, k;
  long long c;
  if (!interior_node(g, i, j, k, c)) return;
  double ya = b.ya[c], yb = b.yb[c], zbw = b.zbw[c], zbv = b.zbv[c];
  bool hya = isfinite(ya), hyb = isfinite(yb);
  double y;
  if (ya < 0.0 && 0.0 < yb) y = 0.0;
  else if (hya && hyb) y = 0.5 * (ya + yb);
  else if (hya) y = ya + 1.0;
  else y = yb - 1.0;
  double w = isfinite(zbw) ? 0.5 * zbw : 1.0;
  double v = isfinite(zbv) ? 0.5 * zbv : 1.0;
  s.y[c] = y;
  s.w[c] = w;
  s.v[c] = v;
  s.p[c] = 0.0;
  s.lya[c] = hya ? mu0 / (y - ya) : 0.0;
  s.lyb[c] = hyb ? mu0 / (yb - y) : 0.0;
  s.lwa[c] = mu0 / w;
  s.lwb[c] = isfinite(zbw) ? mu0 / (zbw - w) : 0.0;
  s.lva[c] = mu0 / v;
  s.lvb[c] = isfinite(zbv) ? mu0 / (zbv - v) : 0.0;
}

// Theta_y, Theta_w, Theta_v; M_hat (cancellation-free form of Section 4.2's
// diagonal: d^2 s / (1 + alpha d s) * (d + theta_y), s = 1/theta_w + 1/theta_v);
// right-hand side of (NewtonSystem) at barrier parameter mu.
__global__ void k_prep(GridDesc g, Stencil<double> st, IpmProblem pb, IpmBounds b, IpmState s,
                       IpmDiag dg, double mu, double* __restrict__ rhs, int write32) {
  int i, j, k;
  long long c;
  if (!interior_node(g, i, j, k, c)) return;
  const long long F = g.field;
  double y = s.y[c], w = s.w[c], v = s.v[c];
  Inv r = inv_dist(b, y, w, v, c);
  double thy = r.ya * s.lya[c] + r.yb * s.lyb[c];
  double thw = r.wa * s.lwa[c] + r.wb * s.lwb[c];
  double thv = r.va * s.lva[c] + r.vb * s.lvb[c];
  double dM = pb.dM;
  double sinv = 1.0 / thw + 1.0 / thv;
  double mh = sqrt(dM * dM * sinv / (1.0 + pb.alpha * dM * sinv) * (dM + thy));
  dg.thy[c] = thy;
  dg.thw[c] = thw;
  dg.thv[c] = thv;
  dg.mh[c] = mh;
  if (write32) {
    dg.thy32[c] = (float)thy;
    dg.mh32[c] = (float)mh;
    dg.thw32[c] = (float)thw;
    dg.thv32[c] = (float)thv;
    const FF t = ff_from_double(thy);
    dg.thyff[c] = t.h;
    dg.thyff[F + c] = t.l;
  }
  double My = st.track(s.y, c);  // tracking mass: M, or M_s under partial observation
  double Mu = st.mass_f(LdDiff<double>{s.w, s.v}, c);
  double Mp = st.mass(s.p, c);
  double Ly = apply_L<double>(pb.L, st, Ld<double>{s.y}, c, F);
  double LTp = apply_LT<double>(pb.L, st, Ld<double>{s.p}, c, F);
  double gy = My - pb.cy[c] + LTp;
  double gw = pb.alpha * Mu + pb.beta * pb.d - Mp;
  double gv = -pb.alpha * Mu + pb.beta * pb.d + Mp;
  double gp = Ly - Mu - pb.fvec[c];
  rhs[c] = -(gy - mu * r.ya + mu * r.yb);
  rhs[F + c] = -(gw - mu * r.wa + mu * r.wb);
  rhs[2 * F + c] = -(gv - mu * r.va + mu * r.vb);
  rhs[3 * F + c] = -gp;
}

IPM_D void ratio_to_bounds(double x, double dx, double lo, double hi, bool hlo, bool hhi,
                           double& a) {
  if (dx < 0.0 && hlo) a = fmin(a, (x - lo) / (-dx));
  if (dx > 0.0 && hhi) a = fmin(a, (hi - x) / dx);
}

struct DLam {
  double ya, yb, wa, wb, va, vb;
};

// (zupdate1)-(zupdate4)
IPM_D DLam mult_steps(const Inv& r, const IpmState& s, long long c, double dy, double dw,
                      double dv, double mu) {
  DLam d;
  double lya = s.lya[c], lyb = s.lyb[c], lwa = s.lwa[c], lwb = s.lwb[c], lva = s.lva[c],
         lvb = s.lvb[c];
  d.ya = r.hya ? (-r.ya * lya * dy - lya + mu * r.ya) : 0.0;
  d.yb = r.hyb ? (r.yb * lyb * dy - lyb + mu * r.yb) : 0.0;
  d.wa = -r.wa * lwa * dw - lwa + mu * r.wa;
  d.wb = r.hwb ? (r.wb * lwb * dw - lwb + mu * r.wb) : 0.0;
  d.va = -r.va * lva * dv - lva + mu * r.va;
  d.vb = r.hvb ? (r.vb * lvb * dv - lvb + mu * r.vb) : 0.0;
  return d;
}

__global__ void k_steplen(GridDesc g, IpmBounds b, IpmState s, const double* __restrict__ dx,
                          double mu, double* __restrict__ part) {
  __shared__ double sh[32];
  int i, j, k;
  long long c;
  bool in = interior_node(g, i, j, k, c);
  double aP = 1e300, aD = 1e300;
  if (in) {
    const long long F = g.field;
    double y = s.y[c], w = s.w[c], v = s.v[c];
    double dy = dx[c], dw = dx[F + c], dv = dx[2 * F + c];
    Inv r = inv_dist(b, y, w, v, c);
    ratio_to_bounds(y, dy, b.ya[c], b.yb[c], r.hya, r.hyb, aP);
    ratio_to_bounds(w, dw, 0.0, b.zbw[c], true, r.hwb, aP);
    ratio_to_bounds(v, dv, 0.0, b.zbv[c], true, r.hvb, aP);
    DLam d = mult_steps(r, s, c, dy, dw, dv, mu);
    if (r.hya && d.ya < 0.0) aD = fmin(aD, s.lya[c] / (-d.ya));
    if (r.hyb && d.yb < 0.0) aD = fmin(aD, s.lyb[c] / (-d.yb));
    if (d.wa < 0.0) aD = fmin(aD, s.lwa[c] / (-d.wa));
    if (r.hwb && d.wb < 0.0) aD = fmin(aD, s.lwb[c] / (-d.wb));
    if (d.va < 0.0) aD = fmin(aD, s.lva[c] / (-d.va));
    if (r.hvb && d.vb < 0.0) aD = fmin(aD, s.lvb[c] / (-d.vb));
  }
  double tP = block_min(aP, sh);
  double tD = block_min(aD, sh);
  if (lin_tid() == 0) {
    long long bi = lin_block();
    part[2 * bi] = tP;
    part[2 * bi + 1] = tD;
  }
}

// alpha_P = alpha_0 min(1, min ratio), alpha_D likewise -> sc[0], sc[1]; with `common`
// both take the smaller value.
__global__ void k_steplen_final(const double* __restrict__ part, long long nb, double alpha0,
                                int common, double* __restrict__ sc) {
  __shared__ double sh[32];
  double aP = 1e300, aD = 1e300;
  for (long long t = threadIdx.x; t < nb; t += blockDim.x) {
    aP = fmin(aP, part[2 * t]);
    aD = fmin(aD, part[2 * t + 1]);
  }
  aP = block_min(aP, sh);
  aD = block_min(aD, sh);
  if (threadIdx.x == 0) {
    double p = alpha0 * fmin(1.0, aP), d = alpha0 * fmin(1.0, aD);
    if (common) p = d = fmin(p, d);
    sc[0] = p;
    sc[1] = d;
  }
}

__global__ void k_update(GridDesc g, IpmBounds b, IpmState s, const double* __restrict__ dx,
                         double mu, const double* __restrict__ sc) {
  int i, j, k;
  long long c;
  if (!interior_node(g, i, j, k, c)) return;
  const long long F = g.field;
  double aP = sc[0], aD = sc[1];
  double y = s.y[c], w = s.w[c], v = s.v[c];
  double dy = dx[c], dw = dx[F + c], dv = dx[2 * F + c], dp = dx[3 * F + c];
  Inv r = inv_dist(b, y, w, v, c);
  DLam d = mult_steps(r, s, c, dy, dw, dv, mu);
  s.y[c] = y + aP * dy;
  s.w[c] = w + aP * dw;
  s.v[c] = v + aP * dv;
  s.p[c] = s.p[c] + aD * dp;
  s.lya[c] = s.lya[c] + aD * d.ya;
  s.lyb[c] = s.lyb[c] + aD * d.yb;
  s.lwa[c] = s.lwa[c] + aD * d.wa;
  s.lwb[c] = s.lwb[c] + aD * d.wb;
  s.lva[c] = s.lva[c] + aD * d.va;
  s.lvb[c] = s.lvb[c] + aD * d.vb;
}

// Per-block sums: ||xi_p||^2, ||xi_d||^2, ||xi_c||^2, sum of complementarity products,
// y^T M y, y^T c_y, u^T M u, 1^T (w + v).
__global__ void k_residuals(GridDesc g, Stencil<double> st, IpmProblem pb, IpmBounds b,
                            IpmState s, double mu, double* __restrict__ part) {
  __shared__ double sh[32];
  int i, j, k;
  long long c;
  bool in = interior_node(g, i, j, k, c);
  double q[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  if (in) {
    const long long F = g.field;
    double y = s.y[c], w = s.w[c], v = s.v[c];
    double My = st.track(s.y, c);
    double Mu = st.mass_f(LdDiff<double>{s.w, s.v}, c);
    double Mp = st.mass(s.p, c);
    double Ly = apply_L<double>(pb.L, st, Ld<double>{s.y}, c, F);
    double LTp = apply_LT<double>(pb.L, st, Ld<double>{s.p}, c, F);
    double gy = My - pb.cy[c] + LTp;
    double gw = pb.alpha * Mu + pb.beta * pb.d - Mp;
    double gv = -pb.alpha * Mu + pb.beta * pb.d + Mp;
    double gp = Ly - Mu - pb.fvec[c];
    double lya = s.lya[c], lyb = s.lyb[c], lwa = s.lwa[c], lwb = s.lwb[c], lva = s.lva[c],
           lvb = s.lvb[c];
    double dy_ = gy - lya + lyb, dw_ = gw - lwa + lwb, dv_ = gv - lva + lvb;
    q[0] = gp * gp;
    q[1] = dy_ * dy_ + dw_ * dw_ + dv_ * dv_;
    double ya = b.ya[c], yb = b.yb[c], zbw = b.zbw[c], zbv = b.zbv[c];
    double pr;
    if (isfinite(ya)) { pr = (y - ya) * lya; q[2] += (pr - mu) * (pr - mu); q[3] += pr; }
    if (isfinite(yb)) { pr = (yb - y) * lyb; q[2] += (pr - mu) * (pr - mu); q[3] += pr; }
    pr = w * lwa; q[2] += (pr - mu) * (pr - mu); q[3] += pr;
    if (isfinite(zbw)) { pr = (zbw - w) * lwb; q[2] += (pr - mu) * (pr - mu); q[3] += pr; }
    pr = v * lva; q[2] += (pr - mu) * (pr - mu); q[3] += pr;
    if (isfinite(zbv)) { pr = (zbv - v) * lvb; q[2] += (pr - mu) * (pr - mu); q[3] += pr; }
    q[4] = y * My;
    q[5] = y * pb.cy[c];
    q[6] = (w - v) * Mu;
    q[7] = w + v;
  }
  long long bi = lin_block();
#pragma unroll
  for (int t = 0; t < 8; ++t) {
    double r = block_sum(q[t], sh);
    if (lin_tid() == 0) part[bi * 8 + t] = r;
  }
}

// [ M + Th_y   0                 0               L^T ] [dy]
// [ 0          alpha M + Th_w    -alpha M        -M  ] [dw]
// [ 0          -alpha M          alpha M + Th_v   M  ] [dv]
// [ L          -M                M                0  ] [dp]
// FP64 output, or (out_ff != null) float-float output: high parts of the four fields,
// then their low parts (a float-float Krylov vector)
__global__ void k_newton_apply(GridDesc g, Stencil<double> st, IpmProblem pb, IpmDiag dg,
                               const double* __restrict__ x, double* __restrict__ out,
                               float* __restrict__ out_ff) {
  int i, j, k;
  long long c;
  if (!interior_node(g, i, j, k, c)) return;
  const long long F = g.field;
  const double* dy = x;
  const double* dw = x + F;
  const double* dv = x + 2 * F;
  const double* dp = x + 3 * F;
  double My = st.track(dy, c);
  double Mp = st.mass(dp, c);
  double Ms = st.mass_f(LdDiff<double>{dw, dv}, c);
  double Ly = apply_L<double>(pb.L, st, Ld<double>{dy}, c, F);
  double LTp = apply_LT<double>(pb.L, st, Ld<double>{dp}, c, F);
  double a = pb.alpha;
  const double r[4] = {My + dg.thy[c] * dy[c] + LTp, a * Ms + dg.thw[c] * dw[c] - Mp,
                       -a * Ms + dg.thv[c] * dv[c] + Mp, Ly - Ms};
  if (out_ff) {
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const FF v = ff_from_double(r[b]);
      out_ff[b * F + c] = v.h;
      out_ff[4 * F + b * F + c] = v.l;
    }
  } else {
#pragma unroll
    for (int b = 0; b < 4; ++b) out[b * F + c] = r[b];
  }
}

// The same operator for the 2D Poisson problem in float-float arithmetic (FP32 pipes; this
// GPU's FP64 rate is ~1/70 of its FP32 rate): a 32 x 8 block stages y, w - v and p of its
// nodes and their one-node halo in shared memory, each FP64 value converted to float-float
// once; the Q1 mass (rows [1 4 1] (x) [1 4 1] times h^2/36) and stiffness (3 x_c minus a
// third of the 3 x 3 box) stencils, the Theta products and the combination run in float-float
// (about 2^-46 relative per operation). Output: float-float Krylov vector planes.
constexpr int kFFX = 32, kFFY = 8;
__global__ void __launch_bounds__(kFFX * kFFY) k_newton_apply_ff2(GridDesc g, FF ms, FF third,
                                                                 FF alpha,
                                                                 const double* __restrict__ x,
                                                                 const float* __restrict__ thyff,
                                                                 const double* __restrict__ thw,
                                                                 const double* __restrict__ thv,
                                                                 float* __restrict__ out) {
  constexpr int SX = kFFX + 2, SY = kFFY + 2;
  __shared__ FF sy[SY][SX], sd[SY][SX], sp[SY][SX];
  const long long F = g.field, p = g.pitch;
  const int X0 = 1 + blockIdx.x * kFFX, Y0 = 1 + blockIdx.y * kFFY;
  const int t = threadIdx.y * kFFX + threadIdx.x;
  for (int q = t; q < SX * SY; q += kFFX * kFFY) {
    const int lx = q % SX, ly = q / SX;
    const int gx = X0 - 1 + lx, gy = Y0 - 1 + ly;
    FF vy{0.f, 0.f}, vd{0.f, 0.f}, vp{0.f, 0.f};
    if (gx < g.n && gy < g.n) {
      const long long c = (long long)gy * p + gx;
      vy = ff_from_double(x[c]);
      vd = ff_from_double(x[F + c] - x[2 * F + c]);
      vp = ff_from_double(x[3 * F + c]);
    }
    sy[ly][lx] = vy;
    sd[ly][lx] = vd;
    sp[ly][lx] = vp;
  }
  __syncthreads();
  const int gx = X0 + threadIdx.x, gy = Y0 + threadIdx.y;
  if (gx > g.n - 2 || gy > g.n - 2) return;
  const int lx = threadIdx.x + 1, ly = threadIdx.y + 1;
  auto four = [](FF a) { return FF{4.f * a.h, 4.f * a.l}; };
  auto mass = [&](FF (*a)[SX]) {
    auto row = [&](int r) { return ff_add(ff_add(a[r][lx - 1], four(a[r][lx])), a[r][lx + 1]); };
    return ff_mul(ms, ff_add(ff_add(row(ly - 1), four(row(ly))), row(ly + 1)));
  };
  auto stiff = [&](FF (*a)[SX]) {
    auto row = [&](int r) { return ff_add(ff_add(a[r][lx - 1], a[r][lx]), a[r][lx + 1]); };
    const FF box = ff_add(ff_add(row(ly - 1), row(ly)), row(ly + 1));
    const FF xc = a[ly][lx];
    // 3 x_c as 2 x_c + x_c: scaling by 2 is exact, by 3 is not
    return ff_add(ff_add(FF{2.f * xc.h, 2.f * xc.l}, xc), ff_neg(ff_mul(third, box)));
  };
  const long long c = (long long)gy * p + gx;
  const FF My = mass(sy), Mp = mass(sp), Md = mass(sd), Ky = stiff(sy), Kp = stiff(sp);
  const FF ty{thyff[c], thyff[F + c]};
  const FF aMd = ff_mul(alpha, Md);
  const FF r0 = ff_add(ff_add(My, ff_mul(ty, sy[ly][lx])), Kp);
  const FF r1 = ff_add(ff_add(aMd, ff_mul(ff_from_double(thw[c]), ff_from_double(x[F + c]))),
                       ff_neg(Mp));
  const FF r2 = ff_add(ff_add(ff_neg(aMd), ff_mul(ff_from_double(thv[c]),
                                                   ff_from_double(x[2 * F + c]))), Mp);
  const FF r3 = ff_add(Ky, ff_neg(Md));
  const FF r[4] = {r0, r1, r2, r3};
#pragma unroll
  for (int b = 0; b < 4; ++b) {
    out[b * F + c] = r[b].h;
    out[4 * F + b * F + c] = r[b].l;
  }
}

// M_hat (and FP32 copies) from given diagonals, as in k_prep
__global__ void k_mhat(GridDesc g, double alpha, double dM, const double* __restrict__ thy,
                       const double* __restrict__ thw, const double* __restrict__ thv,
                       double* __restrict__ mh, float* __restrict__ thy32, float* __restrict__ mh32) {
  int i, j, k;
  long long c;
  if (!interior_node(g, i, j, k, c)) return;
  double sinv = 1.0 / thw[c] + 1.0 / thv[c];
  double m = sqrt(dM * dM * sinv / (1.0 + alpha * dM * sinv) * (dM + thy[c]));
  mh[c] = m;
  thy32[c] = (float)thy[c];
  mh32[c] = (float)m;
}

__global__ void k_to_float2(GridDesc g, const double* __restrict__ a, const double* __restrict__ b,
                            float* __restrict__ a32, float* __restrict__ b32) {
  int i, j, k;
  long long c;
  if (!interior_node(g, i, j, k, c)) return;
  a32[c] = (float)a[c];
  b32[c] = (float)b[c];
}

__global__ void k_reduce_cols(const double* __restrict__ part, long long nrows, int ncols,
                              double* __restrict__ out) {
  __shared__ double sh[32];
  int col = blockIdx.x;
  double acc = 0.0;
  for (long long r = threadIdx.x; r < nrows; r += blockDim.x) acc += part[r * ncols + col];
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0) out[col] = acc;
}

}  // namespace

long long interior_blocks(const GridDesc& g) {
  dim3 gr = interior_grid(g);
  return (long long)gr.x * gr.y * gr.z;
}

static int flat_blocks(const GridDesc& g) {
  long long nn = (long long)g.n * g.n * (g.dim == 3 ? g.n : 1);
  long long b = (nn + 255) / 256;
  return (int)(b < 4096 ? b : 4096);
}

void launch_pack(const GridDesc& g, const double* dense, double* pitched, int mode, cudaStream_t s) {
  count_launches(1);
  k_pack<<<flat_blocks(g), 256, 0, s>>>(g, dense, pitched, mode);
}
void launch_unpack(const GridDesc& g, const double* pitched, const double* bnd, double* dense,
                   cudaStream_t s) {
  count_launches(1);
  k_unpack<<<flat_blocks(g), 256, 0, s>>>(g, pitched, bnd, dense);
}
void launch_setup_data(const GridDesc& g, const double* yd, const double* f, const double* glift,
                       OpL L, double* cy, double* fvec, cudaStream_t s) {
  count_launches(1);
  k_setup_data<<<interior_grid(g), interior_block(), 0, s>>>(g, make_stencil<double>(g), yd, f,
                                                              glift, L, cy, fvec);
}
void launch_element_mass_form(const GridDesc& g, const double* yd, const double* glift,
                              double* part, double* out, cudaStream_t s) {
  count_launches(1);
  k_element_mass_form<<<kRedBlocks, kRedThreads, 0, s>>>(g, yd, glift, part);
  count_launches(1);
  k_reduce_cols<<<1, 256, 0, s>>>(part, kRedBlocks, 1, out);
}
void launch_setup_norms(const GridDesc& g, const double* cy, const double* fvec,
                        const IpmBounds& b, double* part, double* out, cudaStream_t s) {
  count_launches(1);
  k_setup_norms<<<interior_grid(g), interior_block(), 0, s>>>(g, cy, fvec, b, part);
  count_launches(1);
  k_reduce_cols<<<3, 256, 0, s>>>(part, interior_blocks(g), 3, out);
}
void launch_init_state(const GridDesc& g, const IpmBounds& b, IpmState st, double mu0,
                       cudaStream_t s) {
  count_launches(1);
  k_init_state<<<interior_grid(g), interior_block(), 0, s>>>(g, b, st, mu0);
}
void launch_prep(const GridDesc& g, const IpmProblem& pb, const IpmBounds& b, IpmState st,
                 IpmDiag dg, double mu, double* rhs, int write32, cudaStream_t s) {
  count_launches(1);
  k_prep<<<interior_grid(g), interior_block(), 0, s>>>(g, make_stencil<double>(g), pb, b, st, dg,
                                                        mu, rhs, write32);
}
void launch_steplen(const GridDesc& g, const IpmBounds& b, IpmState st, const double* dx,
                    double mu, double alpha0, int common, double* part, double* sc, cudaStream_t s) {
  count_launches(1);
  k_steplen<<<interior_grid(g), interior_block(), 0, s>>>(g, b, st, dx, mu, part);
  count_launches(1);
  k_steplen_final<<<1, 256, 0, s>>>(part, interior_blocks(g), alpha0, common, sc);
}
void launch_update(const GridDesc& g, const IpmBounds& b, IpmState st, const double* dx,
                   double mu, const double* sc, cudaStream_t s) {
  count_launches(1);
  k_update<<<interior_grid(g), interior_block(), 0, s>>>(g, b, st, dx, mu, sc);
}
void launch_residuals(const GridDesc& g, const IpmProblem& pb, const IpmBounds& b, IpmState st,
                      double mu, double* part, double* out, cudaStream_t s) {
  count_launches(1);
  k_residuals<<<interior_grid(g), interior_block(), 0, s>>>(g, make_stencil<double>(g), pb, b, st,
                                                             mu, part);
  count_launches(1);
  k_reduce_cols<<<8, 256, 0, s>>>(part, interior_blocks(g), 8, out);
}
void launch_newton_apply(const GridDesc& g, const IpmProblem& pb, const IpmDiag& dg,
                         const double* x, double* y, cudaStream_t s) {
  count_launches(1);
  k_newton_apply<<<interior_grid(g), interior_block(), 0, s>>>(g, make_stencil<double>(g), pb, dg,
                                                                x, y, nullptr);
}
void launch_newton_apply_ff(const GridDesc& g, const IpmProblem& pb, const IpmDiag& dg,
                            const double* x, float* y, cudaStream_t s) {
  count_launches(1);
  k_newton_apply<<<interior_grid(g), interior_block(), 0, s>>>(g, make_stencil<double>(g), pb, dg,
                                                                x, nullptr, y);
}
void launch_mhat(const GridDesc& g, double alpha, double dM, const double* thy, const double* thw,
                 const double* thv, double* mh, float* thy32, float* mh32, cudaStream_t s) {
  count_launches(1);
  k_mhat<<<interior_grid(g), interior_block(), 0, s>>>(g, alpha, dM, thy, thw, thv, mh, thy32, mh32);
}
void launch_to_float2(const GridDesc& g, const double* a, const double* b, float* a32, float* b32,
                      cudaStream_t s) {
  count_launches(1);
  k_to_float2<<<interior_grid(g), interior_block(), 0, s>>>(g, a, b, a32, b32);
}

static FF ff_from_double_host(double v) {
  const float h = (float)v;
  return FF{h, (float)(v - (double)h)};
}

bool newton_apply_ff2_ok(const GridDesc& g, const IpmProblem& pb) {
  return g.dim == 2 && !g.heat && !g.obs && pb.L.coef == nullptr;
}

void launch_newton_apply_ff2(const GridDesc& g, const IpmProblem& pb, const IpmDiag& dg,
                             const double* x, float* y, cudaStream_t s) {
  const double h2 = g.h * g.h / 36.0;
  const int m = g.n - 2;
  dim3 grid((m + kFFX - 1) / kFFX, (m + kFFY - 1) / kFFY);
  count_launches(1);
  k_newton_apply_ff2<<<grid, dim3(kFFX, kFFY), 0, s>>>(g, ff_from_double_host(h2),
                                                        ff_from_double_host(1.0 / 3.0),
                                                        ff_from_double_host(pb.alpha), x,
                                                        dg.thyff, dg.thw, dg.thv, y);
}
