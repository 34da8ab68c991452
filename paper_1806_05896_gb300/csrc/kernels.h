// Host-side launch wrappers for every device kernel of the library.
//
// All wrappers enqueue on the given stream and return immediately. Pointers
// are device pointers to fields in the pitched full-grid layout of common.cuh.
#pragma once
#include <cuda_runtime.h>
#include <cstddef>
#include "common.cuh"

// Number of kernel launches enqueued by this library since it was loaded.
void count_launches(long long n);
long long launches_total();
long long launches_thread();

// ----------------------------------------------------------------------------
// Problem fields
// ----------------------------------------------------------------------------
struct IpmState {  // primal-dual iterate, FP64
  double *y, *w, *v, *p;
  double *lya, *lyb, *lwa, *lwb, *lva, *lvb;
};
struct IpmBounds {  // +-inf marks an absent bound; the lower bounds of w and v are 0
  const double *ya, *yb, *zbw, *zbv;
};
struct IpmDiag {  // barrier diagonals and the Schur-approximation diagonal M_hat
  double *thy, *thw, *thv, *mh;
  float *thy32, *mh32, *thw32, *thv32;
  float* thyff;  // Theta_y as float-float planes (high parts, then low parts)
};
// Elliptic operator L: Poisson stiffness (stencil == nullptr) or a stored
// 9-point stencil per node (convection-diffusion), coef[o * field + node] =
// L[node, node + offset_o], offsets o = (dy+1)*3 + (dx+1).
struct OpL {
  const double* coef;
  const float* coef32;
};
struct IpmProblem {
  double alpha, beta;
  double dM;  // diag(M), (2h/3)^d
  double d;   // lumped mass, h^d
  const double *cy, *fvec;
  OpL L;
};

// ----------------------------------------------------------------------------
// k_ipm.cu
// ----------------------------------------------------------------------------
void launch_pack(const GridDesc& g, const double* dense, double* pitched, int mode, cudaStream_t s);
void launch_unpack(const GridDesc& g, const double* pitched, const double* bnd, double* dense,
                   cudaStream_t s);
void launch_setup_data(const GridDesc& g, const double* yd, const double* f, const double* glift,
                       OpL L, double* cy, double* fvec, cudaStream_t s);
void launch_element_mass_form(const GridDesc& g, const double* yd, const double* glift,
                              double* part, double* out, cudaStream_t s);
void launch_setup_norms(const GridDesc& g, const double* cy, const double* fvec,
                        const IpmBounds& b, double* part, double* out, cudaStream_t s);
void launch_init_state(const GridDesc& g, const IpmBounds& b, IpmState st, double mu0,
                       cudaStream_t s);
void launch_prep(const GridDesc& g, const IpmProblem& pb, const IpmBounds& b, IpmState st,
                 IpmDiag dg, double mu, double* rhs, int write32, cudaStream_t s);
void launch_steplen(const GridDesc& g, const IpmBounds& b, IpmState st, const double* dx,
                    double mu, double alpha0, int common, double* part, double* sc, cudaStream_t s);
void launch_update(const GridDesc& g, const IpmBounds& b, IpmState st, const double* dx,
                   double mu, const double* sc, cudaStream_t s);
void launch_residuals(const GridDesc& g, const IpmProblem& pb, const IpmBounds& b, IpmState st,
                      double mu, double* part, double* out, cudaStream_t s);
void launch_newton_apply(const GridDesc& g, const IpmProblem& pb, const IpmDiag& dg,
                         const double* x, double* y, cudaStream_t s);
// same operator, output as a float-float Krylov vector (high parts, then low parts)
// the saddle operator evaluated in float-float arithmetic from shared-memory tiles (2D
// Poisson without an observation mask only: newton_apply_ff2_ok); float-float output planes
bool newton_apply_ff2_ok(const GridDesc& g, const IpmProblem& pb);
void launch_newton_apply_ff2(const GridDesc& g, const IpmProblem& pb, const IpmDiag& dg,
                             const double* x, float* y, cudaStream_t s);
void launch_newton_apply_ff(const GridDesc& g, const IpmProblem& pb, const IpmDiag& dg,
                            const double* x, float* y, cudaStream_t s);
long long interior_blocks(const GridDesc& g);

// ----------------------------------------------------------------------------
// k_precond.cu
// ----------------------------------------------------------------------------
template <typename T>
void launch_cheb_init(const GridDesc& g, const double* b, const T* thy, double dM, double inv_theta,
                      T* bT, T* x1, T* x0, cudaStream_t s);
template <typename T, typename To>
void launch_cheb_step(const GridDesc& g, const T* xc, const T* xp, const T* bT, const T* thy,
                      double dM, double omega, double inv_theta, To* out, cudaStream_t s);
void launch_zblock(const GridDesc& g, double adM, const double* rw, const double* rv,
                   const double* thw, const double* thv, double* zw, double* zv, cudaStream_t s);
void launch_zblock32(const GridDesc& g, double adM, const double* rw, const double* rv,
                     const float* thw, const float* thv, double* zw, double* zv, cudaStream_t s);
// float-float P_T pieces (2D Poisson): z-block from FP32 right-hand sides (FP64 results and
// FP32 copies), coupling t = L z_y - M(z_w - z_v) - r_p and (M + Theta_y) s as planes
void launch_zblock32f(const GridDesc& g, double adM, const float* rw, const float* rv,
                      const float* thw, const float* thv, double* zw, double* zv, float* zw32,
                      float* zv32, cudaStream_t s);
void launch_coupling_ff(const GridDesc& g, const float* zy, const float* zw, const float* zv,
                        const float* rph, const float* rpl, float* th, float* tl, cudaStream_t s);
void launch_mass_theta_ff(const GridDesc& g, const float* sh, const float* sl, const float* tyh,
                          const float* tyl, float* oh, float* ol, cudaStream_t s);
template <typename T>
void launch_coupling(const GridDesc& g, OpL L, const double* zy, const double* zw, const double* zv,
                     const double* rp, int triangular, T* t, cudaStream_t s);
template <typename T>
void launch_mass_theta(const GridDesc& g, const T* x, const T* thy, T* out, cudaStream_t s);
// partial observation: diagonals m_l, m_r of the V-cycle operators of S_Pi_hat, and
// out = (M_s + Theta_y) x - r
void launch_pi_diags(const GridDesc& g, double a, double d, const double* thy, const double* thw,
                     const double* thv, double* ml, double* mr, cudaStream_t s);
void launch_track_theta_minus(const GridDesc& g, const double* x, const double* thy,
                              const double* r, double* out, cudaStream_t s);
template <typename Ti, typename To>
void launch_convert(const GridDesc& g, const Ti* x, To* y, cudaStream_t s);

// ----------------------------------------------------------------------------
// k_mg.cu (geometric multigrid on L + diag(m), Galerkin transfer P^T / P)
// ----------------------------------------------------------------------------
template <typename T>
void launch_mg_smooth(const GridDesc& g, OpL L, const T* xin, T* xout, const T* b, const T* m,
                      const T* jinv, int zero_init, int transpose, cudaStream_t s);
template <typename T>
void launch_mg_residual(const GridDesc& g, OpL L, const T* x, const T* b, const T* m, T* r,
                        int transpose, cudaStream_t s);
template <typename T>
void launch_mg_restrict(const GridDesc& gf, const GridDesc& gc, const T* rf, T* bc, cudaStream_t s);
template <typename T>
void launch_mg_prolong_add(const GridDesc& gf, const GridDesc& gc, const T* xc, T* xf,
                           cudaStream_t s);
template <typename T>
void launch_mg_coarsest(const GridDesc& g, OpL L, const T* b, const T* m, T* x, cudaStream_t s);
template <typename T>
void launch_mg_jinv(const GridDesc& g, OpL L, const T* m, double omega, T* jinv, cudaStream_t s);
template <typename T>
void launch_mg_zero(const GridDesc& g, T* x, cudaStream_t s);
void launch_mg_outer(const GridDesc& g, OpL L, const double* xprev, const float* e,
                     const double* b, const double* m, double* xnew, float* r32, int transpose,
                     cudaStream_t s);
// float-float form of the outer step for the 2D Poisson operator (FP32 instruction rates)
void launch_mg_outer_ff(const GridDesc& g, const float* xh_in, const float* xl_in, const float* e,
                        const double* b64, const float* bff, float* b3h, float* b3l,
                        const float* m3h, const float* m3l, float* xh_out, float* xl_out,
                        float* r32, double* out64, float* outff, int first, cudaStream_t s);
void launch_split3_ff(const GridDesc& g, const double* m, float* hi, float* lo, cudaStream_t s);

// ----------------------------------------------------------------------------
// k_mg_fused.cu (2D Poisson: tiled multi-sweep kernels and a one-CTA coarse cycle)
// ----------------------------------------------------------------------------
constexpr int kMaxCoarse = 8;
template <typename T>
struct MGCoarse {  // levels handled inside one CTA, finest first
  int nl;
  int n[kMaxCoarse];
  long long pitch[kMaxCoarse];
  const T* m[kMaxCoarse];
  // general = 0: the Q1 stiffness (8/3 centre, -1/3 neighbours) + diag(m); general = 1: a
  // constant symmetric 9-point stencil per level (centre, edge, corner weights) + diag(m)
  int general;
  T c0[kMaxCoarse], ce[kMaxCoarse], cc[kMaxCoarse];
};
template <typename T>
size_t mg2_coarse_smem(const MGCoarse<T>& cl);
template <typename T>
void launch_mg2_pre_restrict(const GridDesc& g, const GridDesc& gc, const T* xin, T* xout,
                             const T* b, const T* m, T* bc, double omega, int nu, int zero_init,
                             cudaStream_t s);
template <typename T>
void launch_mg2_prolong_post(const GridDesc& g, const GridDesc& gc, const T* xin, const T* xc,
                             T* xout, const T* b, const T* m, double omega, int nu,
                             cudaStream_t s);
template <typename T>
void launch_mg2_coarse(const MGCoarse<T>& cl, const T* btop, T* xtop, double omega, int nu_pre,
                       int nu_post, int load_x, cudaStream_t s);

// Persistent form of the part of an FP32 V-cycle below the finest level (2D Poisson, 5
// smoothing sweeps): one cooperative launch runs the pre-smoothing and restriction of the
// tiled levels (finest first), the one-CTA cycle of the small levels, and the prolongation
// and post-smoothing back up, with grid-wide barriers between the phases. The coarse
// correction equation starts from zero on every level it covers.
constexpr int kMaxMid = 8;
struct MidCycle {
  int nt;                      // tiled levels, finest first
  GridDesc g[kMaxMid + 1];     // g[nt]: top level of the one-CTA part
  float* xa[kMaxMid];          // iterate written by the post-smoothing of level l
  float* xb[kMaxMid];          // scratch iterate: written by the pre-smoothing, read back
  const float* b[kMaxMid];
  const float* m[kMaxMid];
  float* bnext[kMaxMid];       // right-hand side of the next coarser level (restriction)
  MGCoarse<float> cl;          // levels of the one-CTA part (top level: b = bnext[nt - 1])
  float* xcoarse;              // iterate of the one-CTA part's top level
};
// Grid-wide barrier state (zero-initialised device memory, one per stream of use). A block
// that waits longer than a fixed spin budget sets `timeout`, writes NaN to the V-cycle's
// output and leaves, so a failed barrier surfaces as a non-finite Krylov vector.
struct GridBarrier {
  unsigned count;
  unsigned gen;
  int timeout;
  int pad;
};
// Tile-shape autotuning of the FP32 register-blocked pre- and post-smoothing kernels for the
// grid of g: every candidate shape timed on the given buffers (xa, xb, the level's x
// buffers; b, m its right-hand side and diagonal; bc, xc the next coarser level's
// right-hand side and iterate; all overwritten but b, m, xc), the fastest kept for this
// grid size and device for the rest of the process. Returns 0 on success.
int mg2_autotune(const GridDesc& g, const GridDesc& gc, float* xa, float* xb, const float* b,
                 const float* m, float* bc, const float* xc, double omega, cudaStream_t s);
bool mg2_is_tuned(int n);
// Text lines "kernel n=.. dev=..: shape time" of every choice made so far; returns the
// length of the full text (buf may be NULL).
int mg2_tune_report(char* buf, size_t len);
// Pin (shape >= 0) or forget (shape < 0) the choice for kernel 0 (pre) / 1 (post) and grid
// size n on the current device; returns 0, or 1 for an unknown kernel or shape.
int mg2_tune_set(int kernel, int n, int shape);
// Blocks the cooperative launch uses (0: cooperative launches unsupported on this device).
int mg2_mid_blocks(const MidCycle& mc);
void launch_mg2_mid_cycle(const MidCycle& mc, GridBarrier* bar, double omega, int blocks,
                          cudaStream_t s);

// ----------------------------------------------------------------------------
// k_heat.cu (all-at-once heat equation, space-time layout of make_heat_grid)
// ----------------------------------------------------------------------------
// b32 plane k = t plane k + M (plane kp of x32) (kp < 0: t alone); plane kp of x32 -> x64
void launch_heat_plane_rhs(const GridDesc& g, const double* t, int k, int kp, const float* x32,
                           double* x64, float* b32, cudaStream_t s);
void launch_heat_plane_store(const GridDesc& g, int k, const float* x32, double* x64,
                             cudaStream_t s);

// Temporally blocked Chebyshev (2D): `ns` steps per launch with step weights omega[0..ns)
constexpr int kMaxChebBlock = 8;
struct ChebSteps {
  int ns;
  double omega[kMaxChebBlock];
  double gamma;   // 1 / theta
  double dM;      // diag(M)
  double mscale;  // h^2 / 36
};
bool launch_cheb2_rb_f32(const GridDesc& g, const ChebSteps& cs, const float* b, const float* thy,
                         const float* xc_in, const float* xp_in, float* xc_out, float* xp_out,
                         double* final_out, float* final32, int first, cudaStream_t s);
template <typename T, typename Ti, typename To>
void launch_cheb2_block(const GridDesc& g, const ChebSteps& cs, const Ti* b, const T* thy,
                        const T* xc_in, const T* xp_in, T* xc_out, T* xp_out, To* final_out,
                        int first, cudaStream_t s);

// ----------------------------------------------------------------------------
// k_cd.cu (convection-diffusion + SUPG stencil per level)
// ----------------------------------------------------------------------------
void launch_cd_coef(const GridDesc& g, double eps, double* coef, cudaStream_t s);
void launch_to_float(long long n, const double* x, float* y, cudaStream_t s);

// ----------------------------------------------------------------------------
// k_vec.cu (Krylov vector kernels over whole field blocks, deterministic)
// ----------------------------------------------------------------------------
// float-float Krylov vectors (high parts, then low parts; `stride` and `len` in entries)
// (hi = 1: FP32 dots of the high parts only; part needs 4 x kRedBlocks x 8 entries)
void launch_multidot_ff(const float* V, long long stride, int nv, const float* w, long long len,
                        double* part, double* out, float* out_ff, int hi, cudaStream_t s);
// ||w||^2 in FP64 (overflow-safe) and 1/||w|| as a float-float pair
void launch_norm2_ff(const float* w, long long len, double* part, double* out, float* out_ff,
                     cudaStream_t s);
void launch_axpy_multi_ff(float* w, const float* V, long long stride, int nv, const float* coef,
                          double sign, long long len, cudaStream_t s);
void launch_scale_ff(float* v, const float* f, long long len, cudaStream_t s);
void launch_to_ff(float* out, const double* x, double a, long long len, cudaStream_t s);
void launch_from_ff(double* out, const float* v, long long len, cudaStream_t s);
void launch_multidot(const double* V, long long stride, int nv, const double* w, long long len,
                     double* part, double* out, cudaStream_t s);
void launch_axpy_multi(double* w, const double* V, long long stride, int nv, const double* coef,
                       double sign, long long len, cudaStream_t s);
void launch_axpby(double* y, const double* x, double a, double b, long long len, cudaStream_t s);
void launch_dot(const double* a, const double* b, long long len, double* part, double* out,
                cudaStream_t s);
void launch_scale_rsqrt(double* y, const double* x, const double* s, long long len,
                        cudaStream_t st);
void launch_lincomb3(double* y, double a, const double* x1, double b, const double* x2, double c,
                     const double* x3, long long len, cudaStream_t s);
void launch_mhat(const GridDesc& g, double alpha, double dM, const double* thy, const double* thw,
                 const double* thv, double* mh, float* thy32, float* mh32, cudaStream_t s);
// FP32 copies of Theta_w, Theta_v (mixed-precision z-block)
void launch_to_float2(const GridDesc& g, const double* a, const double* b, float* a32, float* b32,
                      cudaStream_t s);
