/*
 * ipm.h -- C ABI of libipm: the interior point method of Pearson, Porcelli and
 * Stoll, "Interior point methods and preconditioning for PDE-constrained
 * optimization problems involving sparsity terms" (2018), on one GB300 GPU.
 *
 * Problem (Section 1, (pb)-(boxs); discrete form (pb_fe)+(boxvector), Section 2):
 *   min  1/2 ||y - y_d||^2_{L2} + alpha/2 ||u||^2_{L2} + beta ||u||_{L1}
 *   s.t. -Lap y = u + f   (or -eps Lap y + w . grad y = u + f, SUPG-stabilised)
 *        y = g on the boundary,  u_a <= u <= u_b,  y_a <= y <= y_b,
 * on the unit square (cube) with Q1 elements on a uniform grid of n nodes per
 * direction. The unknowns are the interior nodes for y, u and p alike.
 * The solver runs Algorithm A.1 (Appendix); each Newton system
 * (NewtonSystem, Section 3) is solved by MINRES with the block-diagonal
 * preconditioner P_D or by (flexible) GMRES with the block-triangular P_T
 * (Section 4), entirely in CUDA kernels.
 *
 * Conventions for every function below:
 *   - Nodal arrays are full grids of n^d doubles, boundary included, C order
 *     with x fastest ("[z][y][x]"). Host pointers unless the name says _device.
 *   - The library copies inputs at call time; the caller keeps ownership of
 *     its buffers. The solver owns all device memory it allocates until
 *     ipm_destroy.
 *   - Every int-returning function returns IPM_OK (0) or one of the IPM_E*
 *     codes; ipm_last_error gives a message. On error nothing is written to
 *     output buffers unless stated.
 *   - A solver is not thread-safe; use one solver per host thread.
 */
#ifndef IPM_H
#define IPM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ipm_solver ipm_solver; /* opaque */

enum {
  IPM_OK = 0,
  IPM_EINVAL = 1,     /* bad argument: grid, alpha <= 0, beta < 0, bounds violating u_a < 0 < u_b */
  IPM_ENOMEM = 2,     /* device allocation failed */
  IPM_ENOTCONV = 3,   /* iteration cap hit; the last iterate is still retrievable */
  IPM_EBREAKDOWN = 4, /* Krylov breakdown or non-finite values */
  IPM_ETIMEOUT = 5,   /* wall-clock limit of ipm_options.time_limit_s reached */
  IPM_ECUDA = 6,      /* CUDA runtime error */
  IPM_ESTATE = 7      /* call out of order (e.g. solve before set_data, get before solve) */
};

/* Grid: dim = 2 or 3, n[0] = n[1] (= n[2]) = nodes per direction incl. boundary,
 * n = 2^k + 1 with k >= 1 (the multigrid hierarchy halves the mesh down to 3 nodes). */
typedef struct {
  int dim;
  int n[3];
} ipm_grid;

/* State equation: Poisson (Sections 5.1), convection-diffusion with SUPG
 * (Section 5.2; 2D only) with diffusion eps and the recirculating wind
 * w = (2 x2 (1 - x1^2), -2 x1 (1 - x2^2)) (wind = 0), or the heat equation
 * y_t - Lap y = u + f on (0, T) (Section 3.4, all-at-once, backward Euler).
 * IPM_HEAT: grid dim = 2 with n <= 65 nodes per direction; the time interval (0, T)
 * is split into n - 2 steps of tau = T / (n - 2), so every nodal array holds n^3 values:
 * n^2 per time level t_0 = 0, t_1, ..., t_{n-2} = T, then one unused level. The Dirichlet
 * data g carries the initial state y_0 in level 0 (its other entries must be zero); y_d,
 * f, the bounds and the results use levels 1 .. n-2. The cost and the L1 term integrate
 * in time by the rectangle rule; no state bounds; GMRES + P_T only. */
typedef enum { IPM_POISSON = 0, IPM_CONVDIFF_SUPG = 1, IPM_HEAT = 2 } ipm_pde_kind;
typedef struct {
  int kind;
  double eps;
  int wind;
  double T; /* final time (IPM_HEAT) */
} ipm_pde;

/* Bounds (Section 1, (box), (boxs)). Scalars, or nodal arrays when the pointer
 * is non-NULL (full grid, only interior entries are read). The control bounds
 * must satisfy u_a < 0 < u_b (the paper's sign convention) and may be +-INFINITY;
 * y_a = -INFINITY / y_b = +INFINITY mark an absent state bound. */
typedef struct {
  double ua, ub, ya, yb;
  const double *ua_v, *ub_v, *ya_v, *yb_v;
} ipm_bounds;

enum { IPM_PREC_FP64 = 0, IPM_PREC_MIXED = 1 };
enum { IPM_KRYLOV_MINRES_PD = 0, IPM_KRYLOV_GMRES_PT = 1 };
enum { IPM_STOP_PAPER = 0, IPM_STOP_KKT = 1, IPM_STOP_FIXED = 2 };

/* Partial observation (the subsection "Preconditioner for Partial Observations",
 * Section 4): the tracking term 1/2 ||y - y_d||^2 integrates only over the elements whose
 * centre lies strictly inside the box lo < x < hi (dim values each; the third is ignored
 * in 2D), so the state row of (NewtonSystem) carries the singular mass M_s of the observed
 * elements, and GMRES is preconditioned with P_Pi (three solves with L, L^T + M_l and
 * L + M_r, Section 4), in FP64. lo = hi = NULL restores observation of the whole domain.
 * Must precede ipm_set_data. IPM_EINVAL for a box with no element, or for the heat
 * equation. Declared with the other solver calls below. */

/* Solver options; ipm_default_options fills the paper's values (Section 5):
 * alpha0 = 0.995, eps_p = eps_d = eps_c = 1e-6, sigma = 0.2, mu0 = 1,
 * Krylov tolerance 1e-10 (relative unpreconditioned residual), 20 Chebyshev
 * steps, 3 V-cycles with 5 pre- and 5 post-smoothing steps.
 *   precision: IPM_PREC_FP64 everywhere, or IPM_PREC_MIXED (Chebyshev and
 *              multigrid in FP32; the IPM, the true residuals and the Krylov scalars in
 *              FP64; GMRES is then flexible GMRES, and for 2D Poisson without partial
 *              observation its Arnoldi basis, orthogonalisation and saddle operator use
 *              float-float arithmetic (two floats per value, about 2^-46 relative per
 *              operation; kernel_flags bits 5 and 10 select FP64 instead); MINRES runs
 *              inside an FP64 iterative refinement loop that restores krylov_tol on the
 *              true residual).
 *   krylov:    IPM_KRYLOV_MINRES_PD (MINRES + P_D) or IPM_KRYLOV_GMRES_PT
 *              (GMRES + P_T, right-preconditioned, flexible form).
 *   stop:      IPM_STOP_PAPER: ||xi_p|| <= eps_p, ||xi_d|| <= eps_d, ||xi_c|| <= eps_c
 *              (Algorithm A.1); IPM_STOP_KKT: kkt_rel <= kkt_tol; IPM_STOP_FIXED:
 *              exactly fixed_iters IPM iterations.
 *   kkt_rel = max( ||xi_p|| / (1 + ||f|| + ||M y_d||), ||xi_d|| / (1 + ||M y_d|| + beta ||D 1||),
 *                  mean complementarity product / (1 + |Q(y, z)|) ).
 *   common_step, mu_rule: variants of Algorithm A.1's step-length and barrier
 *              updates (defaults 0 = as printed in the paper).                          */
typedef struct {
  int precision;
  int krylov;
  int stop;
  double sigma, alpha0, eps_p, eps_d, eps_c, mu0, kkt_tol, krylov_tol;
  int cheb_steps, vcycles, smooth_pre, smooth_post;
  int max_ipm, max_krylov, restart, fixed_iters;
  double time_limit_s; /* <= 0: none */
  int common_step; /* 0: separate alpha_P, alpha_D (Algorithm A.1); 1: both = min(alpha_P, alpha_D) */
  int mu_rule;     /* 0: mu <- sigma mu (Algorithm A.1); 1: mu <- sigma * mean complementarity product */
  int kernel_flags; /* 0: fastest kernels; bit 0: per-sweep multigrid/Chebyshev kernels instead of
                       the fused 2D ones; bit 1: no CUDA-graph replay of Krylov iterations;
                       bits 2 / 3: on the mixed path keep the Chebyshev and z-block / the
                       multigrid stage in FP64;
                       bit 4: mixed multigrid on the 2D Poisson operator takes its finest-level
                       outer residual in FP64 instead of float-float arithmetic;
                       bit 5: mixed FGMRES keeps its Arnoldi basis in FP64 instead of
                       float-float (orthogonalisation and norms); bit 6: with a float-float
                       basis, apply P_T to its FP64 conversion instead of in float-float;
                       bit 7: run the FP32 multigrid levels from 129^2 down as one persistent
                       cooperative launch per V-cycle instead of one launch per level (same
                       results to FP32 accuracy; fewer launches, no faster on GB300);
                       bit 8: mixed-precision MINRES without its FP64 iterative refinement;
                       bit 9: no tile-shape autotuning (the fixed shapes of a timing sweep);
                       bit 10: mixed FGMRES evaluates the saddle operator in FP64 instead of
                       float-float */
} ipm_options;

typedef struct {
  int status;             /* IPM_OK, IPM_ENOTCONV, ... */
  int ipm_iters;          /* Newton steps taken */
  int krylov_iters_total; /* Krylov iterations over all Newton steps */
  double kkt_rel, xi_p, xi_d, xi_c, mu;
  double krylov_relres_max; /* worst final relative residual of the Newton solves */
  double seconds;           /* wall time of ipm_solve */
} ipm_report;

void ipm_default_options(ipm_options* opt);

/* Create a solver for one problem on the current CUDA device: allocates the nodal
 * fields, both multigrid hierarchies and the solver's own stream; the Krylov basis is
 * allocated by the first solve that needs it (and grows with a larger restart).
 * beta >= 0, alpha > 0. On success *out owns the solver. */
int ipm_create(const ipm_grid* grid, const ipm_pde* pde, double alpha, double beta,
               const ipm_bounds* bounds, ipm_solver** out);

/* Reuse a solver for a new problem on the same grid and state equation: new alpha, beta
 * and bounds (validated as in ipm_create); ipm_set_data must follow before ipm_solve.
 * Keeps all device memory. */
int ipm_reset(ipm_solver* s, double alpha, double beta, const ipm_bounds* bounds);

/* Device memory owned by the solver, in bytes (grows when a solve needs a larger
 * Krylov basis). */
size_t ipm_device_bytes(const ipm_solver* s);

/* Use an existing CUDA stream (cudaStream_t passed as void*; NULL = the
 * solver's own stream). All device work of later calls is ordered on it. When the
 * stream changes, the call first waits on the host for the work already enqueued on
 * the previous one. Returns IPM_ECUDA if that wait reports an error. */
int ipm_set_stream(ipm_solver* s, void* cuda_stream);

int ipm_set_observation(ipm_solver* s, const double* lo, const double* hi);

/* Problem data (Section 1): desired state y_d, source f, Dirichlet data g
 * (boundary entries of g are used). Host arrays of n^d doubles; NULL = zero. */
int ipm_set_data(ipm_solver* s, const double* yd, const double* f, const double* g);
/* Same, from device arrays of n^d doubles (no host copy). */
int ipm_set_data_device(ipm_solver* s, const double* yd, const double* f, const double* g);

/* Run Algorithm A.1 from the central-path start. opt NULL = defaults; rep may be
 * NULL. Returns IPM_OK or IPM_ENOTCONV (iterate still available), or an error. */
int ipm_solve(ipm_solver* s, const ipm_options* opt, ipm_report* rep);

/* Results after ipm_solve into caller-owned buffers of len = n^d doubles:
 * state y (boundary = g), control u = w - v (boundary 0), adjoint p (boundary 0). */
int ipm_get_state(const ipm_solver* s, double* y, size_t len);
int ipm_get_control(const ipm_solver* s, double* u, size_t len);
int ipm_get_adjoint(const ipm_solver* s, double* p, size_t len);
/* Same into device buffers of n^d doubles (enqueued on the solver's stream). */
int ipm_get_state_device(const ipm_solver* s, double* y, size_t len);
int ipm_get_control_device(const ipm_solver* s, double* u, size_t len);
int ipm_get_adjoint_device(const ipm_solver* s, double* p, size_t len);

/* Per-iteration history of the last solve: rows of 10 doubles
 * (k, mu, ||xi_p||, ||xi_d||, ||xi_c||, kkt_rel, alpha_P, alpha_D, krylov_iters,
 *  krylov_relres); row 0 is the starting point. Writes min(max_rows, rows). */
int ipm_get_history(const ipm_solver* s, double* rows, int max_rows, int* n_rows);

void ipm_destroy(ipm_solver* s);
/* Total number of CUDA kernels this library has launched since it was loaded
 * (all solvers, all threads). */
long long ipm_launch_count(void);
/* Sampled timing of the finest-level multigrid smoother (the dominant kernel):
 * enable = 1 starts recording a CUDA event pair around every `every`-th launch on
 * the solver's stream (and clears earlier samples); enable = 0 stops.
 * ipm_profile_read returns the summed event time of the sampled launches, their
 * number, and the average algorithmic bytes one sampled launch moves per the values it
 * reads and writes once per unknown (fused 2D kernel: x (unless it starts from zero), b, m
 * read, x and a quarter-size coarse right-hand side written; per-sweep kernel: x, b, m,
 * jinv read, x written), in the precision of the last solve. */
int ipm_profile_smoother(ipm_solver* s, int enable, int every);
int ipm_profile_read(ipm_solver* s, double* total_ms, long long* launches, double* bytes_per_launch);
/* The same sampling for one of several kernels of the 2D fused multigrid path and the
 * Krylov iteration: kind 0 the finest-level pre-smoothing + restriction, 1 the finest-level
 * prolongation + post-smoothing, 2 the one-CTA coarse cycle (or, with kernel_flags bit 7,
 * the persistent cycle from 129^2 down), 3 the saddle operator of (NewtonSystem), 4 the
 * tiled launches of the levels between the finest and the coarse cycle.
 * ipm_profile_kernel_read returns the summed event time of the sampled launches, their
 * number, the number of launches of that kind since enabling (sampled or not), and the
 * average algorithmic bytes of a sampled launch counted two ways: bytes_pass, every sweep
 * or pass reading its operands and writing its result once (the per-pass count of a
 * stencil sweep); bytes_once, every value a launch needs read or written once (what a
 * temporally blocked kernel moves at best). */
int ipm_profile_kernel(ipm_solver* s, int kind, int enable, int every);
int ipm_profile_kernel_read(ipm_solver* s, double* total_ms, long long* sampled, long long* calls,
                            double* bytes_pass, double* bytes_once);
/* Per-stage CUDA-event timing of the Krylov iteration (disables graph replay while on).
 * Copies the accumulated milliseconds and counts of up to `nphases` stages into ms /
 * counts (stages: 1 Chebyshev, 2 z-block + coupling, 3 multigrid solves, 4 (M + Theta_y)
 * product and conversion, 5 normalisation and norm, 6 Newton operator, 7 Gram-Schmidt
 * dot products, 8 Gram-Schmidt updates; inside the 2D multigrid: 9 finest-level pre-smoothing
 * + restriction, 10 finest-level prolongation + post-smoothing, 11 the other tiled levels,
 * 12 the one-CTA coarse cycle), then, if enable >= 0, resets them and switches
 * stage timing on (1) or off (0). */
int ipm_profile_phases(ipm_solver* s, int enable, double* ms, long long* counts, int nphases);
/* Tile shapes chosen so far by the autotuner of the FP32 multigrid kernels (the first
 * mixed-precision solve on a grid size times every candidate shape once per process and
 * device; shapes change timing only, not results): text lines "kernel n=.. dev=..: shape
 * time" into buf (len bytes, NUL-terminated, may be NULL); returns the full text length. */
int ipm_tuning_report(char* buf, size_t len);
/* Pin the tile shape of kernel 0 (pre-smoothing + restriction) or 1 (prolongation +
 * post-smoothing) for grid size n on the current device (shape = index into the
 * candidates: pre 52x52/16w, 20x32/8w, 52x32/8w, 52x24/8w, 20x64/8w, 20x18/8w, 20x36/16w;
 * post 56x32/8w, 24x24/8w, 56x56/16w, 24x48/8w, 56x24/8w, 24x16/8w, 24x40/16w), or forget
 * it (shape < 0) so that the next solve
 * tunes again. For reproducible kernel selection. IPM_EINVAL for an unknown kernel/shape. */
int ipm_tuning_set(int kernel, int n, int shape);
const char* ipm_strerror(int code);
const char* ipm_last_error(const ipm_solver* s);

/* ---------------------------------------------------------------------------
 * Serving: independent solves of many requests on one GPU. Worker threads each own a
 * CUDA stream, so requests overlap on the device; a request is admitted when its solver
 * fits the device-memory budget (solvers are pooled per grid and state equation, reset
 * per request, and idle ones are evicted when another grid needs room). Results do not
 * depend on what else runs: every kernel's reductions have a fixed order.
 * --------------------------------------------------------------------------- */
typedef struct ipm_server ipm_server;
typedef struct {
  ipm_grid grid;
  ipm_pde pde;
  double alpha, beta;
  ipm_bounds bounds; /* scalar bounds only (nodal arrays are rejected) */
  const double* yd;  /* host, n^d doubles, copied at submission */
  ipm_options opt;
} ipm_request;

/* Start `workers` worker threads on the current device with a device-memory budget. */
int ipm_server_create(int workers, size_t hbm_budget_bytes, ipm_server** out);
/* Queue a request (returns at once). IPM_ENOMEM if it can never fit the budget. */
int ipm_server_submit(ipm_server* sv, const ipm_request* rq, long long* ticket);
/* Block until the request is done; copy its report and control (len = n^d doubles, may be
 * NULL), its latency from submission to completion and its time in the queue (seconds).
 * Returns the solve's status. A ticket can be waited for once. */
int ipm_server_wait(ipm_server* sv, long long ticket, ipm_report* rep, double* u, size_t len,
                    double* latency_s, double* queue_s);
int ipm_server_stats(ipm_server* sv, size_t* bytes_in_use, int* solvers, long long* completed);
/* Stop the workers (after the running solves) and free every pooled solver. Queued
 * requests that have not started are dropped with their tickets: call it only when no
 * thread is blocked in, or will still call, ipm_server_wait. */
void ipm_server_destroy(ipm_server* sv);

/* ---------------------------------------------------------------------------
 * Component entry points: one stage of the hot path on device buffers, for
 * checking kernels in isolation. Nodal device arrays of n^d doubles (dense,
 * boundary included, x fastest); "4-field" arrays hold (y, w, v, p) blocks of
 * n^d each, back to back. Boundary entries of inputs are ignored, outputs get
 * zero boundaries. They use the solver's grid, operator and parameters.
 * --------------------------------------------------------------------------- */

/* out = calA x with calA the matrix of (NewtonSystem) for the given diagonals
 * Theta_y, Theta_w, Theta_v (Section 3). x, out: 4-field. */
int ipm_newton_apply_device(ipm_solver* s, const double* theta_y, const double* theta_w,
                            const double* theta_v, const double* x, double* out);

/* The same product evaluated as on the mixed-precision FGMRES path: in float-float
 * arithmetic (two floats per value, about 2^-46 relative per operation) from shared-memory
 * tiles, for the 2D Poisson problem without partial observation (IPM_EINVAL otherwise);
 * the float-float result is returned as FP64 (high + low parts). */
int ipm_newton_apply_ff_device(ipm_solver* s, const double* theta_y, const double* theta_w,
                               const double* theta_v, const double* x, double* out);

/* z = P^{-1} r for P_D (triangular = 0) or P_T (triangular = 1) built from the
 * given diagonals (Section 4), with the options' Chebyshev / multigrid settings
 * and precision. r, z: 4-field. */
int ipm_precond_apply_device(ipm_solver* s, const ipm_options* opt, int triangular,
                             const double* theta_y, const double* theta_w, const double* theta_v,
                             const double* r, double* z);

/* x = Chebyshev_k(M + Theta_y)^{-1} b: k steps of Chebyshev semi-iteration with
 * the Jacobi splitting D_M + Theta_y (Section 4.1), FP64. b, x: nodal. */
int ipm_chebyshev_device(ipm_solver* s, int steps, const double* theta_y, const double* b,
                         double* x);

/* x = V-cycle approximation of (L + diag(m))^{-1} b (transpose = 1: (L^T + diag(m))^{-1}),
 * `vcycles` V-cycles from x = 0 with the options' smoothing counts. m, b, x: nodal.
 * FP64 unless opt->precision is IPM_PREC_MIXED: then the cycles run in FP32 on the
 * correction equation with an FP64 residual and iterate on the finest level, as inside
 * the mixed-precision preconditioner. */
int ipm_vcycle_device(ipm_solver* s, const ipm_options* opt, int transpose, const double* m,
                      const double* b, double* x);

/* Newton direction of Algorithm A.1 from a given iterate: loads (y, w, v, p and
 * the six multipliers; 10 nodal arrays, NULL multipliers for absent bounds), forms
 * Theta, M_hat and the right-hand side at barrier parameter mu, and solves
 * (NewtonSystem) with the options' Krylov method. dx: 4-field output. Also
 * returns the Krylov iteration count and final relative residual when non-NULL. */
int ipm_newton_step_device(ipm_solver* s, const ipm_options* opt, const double* const* iterate,
                           double mu, double* dx, int* iters, double* relres);

/* Allocation-free Chebyshev semi-iteration (the paper has no counterpart: this
 * entry point exists for callers that cannot let a library call cudaMalloc, e.g.
 * applications that hand out all device memory from their own pool, or service
 * loops where an allocation and the synchronisation it may imply would stall
 * other work). Same result as ipm_chebyshev_device: x = `steps` steps of
 * Chebyshev semi-iteration for (M + Theta_y) x = b on the Q1 grid of n^dim nodes,
 * FP64. theta_y, b, x: device arrays of n^dim doubles (dense, boundary included,
 * x fastest); x gets a zero boundary and must not alias theta_y or b. Work is
 * enqueued on `stream` (NULL = legacy default stream).
 * Work vectors live in one fixed device array of 3 * 274625 doubles (6.3 MiB)
 * that every GPU loading the library keeps until the process exits (with lazy
 * module loading, the default, the array is materialised on a device by the
 * first call there, not at library load); grids with n^dim > 274625 (beyond
 * 65^3, 513^2) are rejected with IPM_EINVAL. The first call on a device (and
 * the first after a device reset) looks up that array's device address
 * (cudaGetSymbolAddress) with the device current; make that first call before
 * any stream capture.
 * All calls share the array and each clears the part it uses: calls that overlap
 * on the GPU (different streams, or host threads racing) corrupt each other.
 * No cudaMalloc, cudaFree or allocating library routine is called. */
int ipm_chebyshev_noalloc(int dim, int n, int steps, const double* theta_y, const double* b,
                          double* x, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* IPM_H */
