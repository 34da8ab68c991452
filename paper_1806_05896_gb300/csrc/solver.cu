// Host orchestration of the interior point method (Algorithm A.1, Appendix)
// with preconditioned Krylov solves of (NewtonSystem) (Sections 3-4), and the
// C ABI declared in include/ipm.h. Every arithmetic step runs in the kernels of
// k_*.cu; the host only sequences launches and reads back scalars.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <string>
#include <type_traits>
#include <vector>

#include "ipm.h"
#include "kernels.h"

namespace {

struct IpmError {
  int code;
  std::string msg;
};

#define CK(call)                                                                     \
  do {                                                                               \
    cudaError_t e_ = (call);                                                         \
    if (e_ != cudaSuccess)                                                           \
      throw IpmError{IPM_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)}; \
  } while (0)

constexpr int kMaxRestart = 100;
constexpr int kHistCols = 10;

template <typename T>
struct MGLevel {
  GridDesc g;
  T* x[2];
  T* b;
  T* r;
  T* m;
  T* jinv;
};
template <typename T>
struct MGHier {
  int nlev = 0;
  MGLevel<T> lv[16];
  int cur[16];
};

}  // namespace

struct ipm_solver {
  GridDesc g;
  ipm_pde pde;
  double alpha = 0, beta = 0;
  cudaStream_t stream = nullptr;
  cudaStream_t own = nullptr;
  std::vector<void*> allocs;
  std::vector<size_t> alloc_bytes;  // size of each entry of allocs
  size_t bytes = 0;

  IpmState st{};
  double *ya = nullptr, *yb = nullptr, *zbw = nullptr, *zbv = nullptr;
  double *cy = nullptr, *fvec = nullptr, *glift = nullptr;
  double *ydbuf = nullptr, *fbuf = nullptr;  // packed nodal y_d and f (boundary included)
  IpmDiag dg{};
  double *rhs = nullptr, *dx = nullptr, *ktmp = nullptr;
  double *V = nullptr, *Z = nullptr;
  int vcap = 0;
  // float-float Arnoldi basis (mixed precision): V_j holds high parts then low parts;
  // kff holds the Gram-Schmidt coefficients and 1/||w|| as float-float pairs
  bool krylov_ff = false;
  float* kff = nullptr;
  // layout of the basis entries the kernels never write (boundary and padding nodes, which
  // must read as zero): -1 all zero, 0 FP64, 1 float-float
  int vlayout = -1;
  double* mr[16] = {};
  double* cheb64[4] = {};
  float* cheb32[4] = {};
  MGHier<double> mg64;
  MGHier<float> mg32;
  double *mgb64 = nullptr, *mgx64[2] = {};  // FP64 right-hand side and iterates of the mixed solve
  float *mgb3 = nullptr, *mgm3 = nullptr;    // float-float 3b and 3m (high part, then low part)
  float* mgxf[2] = {};                       // float-float iterates (own buffers: the FP64 ones
                                             // keep zero boundaries in their own layout)
  float* zf32 = nullptr;                     // FP32 copies of z_y, z_w, z_v (float-float P_T)
  float* pff[3] = {};                        // float-float planes: t, S^{-1}-stage iterate, rhs
  bool ff_outer = true;
  // stored operator per multigrid level (convection-diffusion); empty for Poisson
  std::vector<OpL> lvop;
  double *part = nullptr, *dout = nullptr, *sc = nullptr, *kdev = nullptr;
  long long part_rows = 0;
  double* hbuf = nullptr;  // pinned
  double* dense = nullptr; // n^d scratch for packing

  // sampled CUDA-event timing of the finest-level smoother launches (phase 0), and
  // with phase timing on, of every stage of the Krylov iteration (phases 1..)
  bool prof_on = false;
  bool phases_on = false;
  int prof_every = 8;
  long long prof_seen = 0;
  std::vector<cudaEvent_t> prof_ev;
  std::vector<int> prof_tag;
  std::vector<double> prof_bp, prof_bo;  // algorithmic bytes of each sampled launch
  double prof_bp_sum = 0.0, prof_bo_sum = 0.0;
  int prof_used = 0;
  double prof_ms = 0.0;
  long long prof_count = 0;
  long long prof_zero = 0;  // sampled launches that started from a zero iterate
  double ph_ms[16] = {};
  long long ph_count[16] = {};

  double c0 = 0, ncy = 0, nf = 0, nd = 0, nbounds = 0;
  double mean_prod = 0;  // mean complementarity product of the current iterate
  bool has_data = false, solved = false;
  bool fused = true;  // use the fused 2D multigrid kernels
  int last_precision = IPM_PREC_MIXED;
  // CUDA graphs of the FGMRES iteration body, one per Arnoldi index j, for one
  // configuration key (precision, preconditioner, smoothing, stream); a body is
  // captured the second time it runs (its first, eager run sets kernel attributes)
  bool use_graphs = true;
  std::vector<cudaGraphExec_t> gexec;
  std::vector<int> gruns;
  long long gkey = -1;
  std::vector<double> hist;  // rows of kHistCols
  std::string err;

  long long F() const { return g.field; }
  long long nn() const { return (long long)g.n * g.n * (g.dim == 3 ? g.n : 1); }
  long long nI() const {
    long long m = g.n - 2;
    return g.dim == 3 ? m * m * m : m * m;
  }

  template <typename T>
  T* alloc(long long count) {
    void* p = nullptr;
    size_t b = (size_t)count * sizeof(T);
    cudaError_t e = cudaMalloc(&p, b);
    if (e != cudaSuccess) {
      cudaGetLastError();
      throw IpmError{IPM_ENOMEM, "cudaMalloc of " + std::to_string(b) + " bytes failed"};
    }
    allocs.push_back(p);
    alloc_bytes.push_back(b);
    bytes += b;
    // zeroed on the solver's stream: the streams are non-blocking, so a memset on the
    // legacy stream would not be ordered before this solver's kernels (buffers are also
    // allocated in the middle of a solve, when the Krylov basis grows)
    CK(cudaMemsetAsync(p, 0, b, stream));
    return (T*)p;
  }
  void prof_flush() {
    if (prof_used == 0) return;
    CK(cudaStreamSynchronize(stream));
    for (int i = 0; i + 1 < prof_used; i += 2) {
      float ms = 0.f;
      CK(cudaEventElapsedTime(&ms, prof_ev[i], prof_ev[i + 1]));
      int tag = prof_tag[i / 2];
      if (tag == 0 || tag >= 13) {
        prof_ms += ms;
        ++prof_count;
        if (tag == 13) ++prof_zero;
        prof_bp_sum += prof_bp[i / 2];
        prof_bo_sum += prof_bo[i / 2];
      } else {
        ph_ms[tag] += ms;
        ++ph_count[tag];
      }
    }
    prof_used = 0;
  }
  void ensure_events() {
    if (prof_ev.size() < 8192) {
      while (prof_ev.size() < 8192) {
        cudaEvent_t e;
        CK(cudaEventCreate(&e));
        prof_ev.push_back(e);
      }
      prof_tag.assign(4096, 0);
      prof_bp.assign(4096, 0.0);
      prof_bo.assign(4096, 0.0);
    }
  }
  int prof_open = 0;  // event pairs begun but not yet ended
  // event pair around a stage: the slot is reserved at begin, so stages may nest;
  // returns -1 when timing is off or the pool is full
  int ph_begin(int tag) {
    if (!phases_on) return -1;
    ensure_events();
    if (prof_used + 2 > (int)prof_ev.size() && prof_open == 0) prof_flush();
    if (prof_used + 2 > (int)prof_ev.size()) return -1;
    int slot = prof_used;
    prof_used += 2;
    ++prof_open;
    prof_tag[slot / 2] = tag;
    CK(cudaEventRecord(prof_ev[slot], stream));
    return slot;
  }
  void ph_end(int slot) {
    if (slot < 0) return;
    CK(cudaEventRecord(prof_ev[slot + 1], stream));
    --prof_open;
  }
  // sampled smoother timing (tag 0; tag 13 for launches that start from a zero iterate)
  // kernel sampled by the profile hook: 0 finest-level pre-smoothing + restriction,
  // 1 finest-level prolongation + post-smoothing, 2 persistent cycle below the finest level,
  // 3 saddle operator
  int prof_kind = 0;
  // bp, bo: algorithmic bytes of the launch, per pass and once (ipm_profile_kernel_read)
  int prof_begin_kind(int kind, int tag, double bp = 0.0, double bo = 0.0) {
    if (kind != prof_kind) return -1;
    int slot = prof_begin(tag);
    if (slot >= 0) {
      prof_bp[slot / 2] = bp;
      prof_bo[slot / 2] = bo;
    }
    return slot;
  }
  // algorithmic bytes of the FP32 2D multigrid launches, from the unknowns of a level:
  // a sweep reads x, b, M_hat and writes x (4 values per pass); the residual and
  // restriction read x, b, M_hat and write the coarse right-hand side (4); prolongation
  // and correction read x and the coarse x and write x (3). "Once": every value a launch
  // needs, read or written once.
  static double u2(int n) { return (double)(n - 2) * (n - 2); }
  static double pre_pass(int n, int nu, bool zero) { return (4.0 * nu + 4.0 - zero) * u2(n) * 4; }
  static double pre_once(int n, bool zero) { return (4.25 - zero) * u2(n) * 4; }
  static double post_pass(int n, int nu) { return (3.0 + 4.0 * nu) * u2(n) * 4; }
  static double post_once(int n) { return 4.25 * u2(n) * 4; }
  int prof_begin(int tag = 0) {
    if (!prof_on || phases_on || (prof_seen++ % prof_every) != 0) return -1;
    ensure_events();
    if (prof_used + 2 > (int)prof_ev.size() && prof_open == 0) prof_flush();
    if (prof_used + 2 > (int)prof_ev.size()) return -1;
    int slot = prof_used;
    prof_used += 2;
    ++prof_open;
    prof_tag[slot / 2] = tag;
    CK(cudaEventRecord(prof_ev[slot], stream));
    return slot;
  }
  void prof_end(int slot) { ph_end(slot); }

  void drop_graphs() {
    for (cudaGraphExec_t e : gexec)
      if (e) cudaGraphExecDestroy(e);
    gexec.clear();
    gruns.clear();
    gcount.clear();
  }

  void release() {
    drop_graphs();
    for (cudaEvent_t e : prof_ev) cudaEventDestroy(e);
    prof_ev.clear();
    for (void* p : allocs) cudaFree(p);
    allocs.clear();
    alloc_bytes.clear();
    if (hbuf) cudaFreeHost(hbuf);
    hbuf = nullptr;
    if (own) cudaStreamDestroy(own);
    own = nullptr;
  }

  OpL opL() const { return lvop.empty() ? OpL{nullptr, nullptr} : lvop[0]; }
  OpL opl(int l) const { return lvop.empty() ? OpL{nullptr, nullptr} : lvop[l]; }
  IpmProblem problem() const {
    IpmProblem pb;
    pb.alpha = alpha;
    pb.beta = beta;
    pb.dM = mass_diag(g);
    pb.d = lumped_mass(g);
    pb.cy = cy;
    pb.fvec = fvec;
    pb.L = opL();
    return pb;
  }
  IpmBounds bounds() const { return IpmBounds{ya, yb, zbw, zbv}; }
  double omega() const { return g.dim == 2 ? 8.0 / 9.0 : 0.95; }

  void sync() {
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(stream));
  }
  void fetch(const double* dsrc, int count) {
    CK(cudaMemcpyAsync(hbuf, dsrc, sizeof(double) * count, cudaMemcpyDeviceToHost, stream));
    sync();
  }

  // ------------------------------------------------------------------------
  template <typename T>
  void build_mg(MGHier<T>& mg) {
    int n = g.n;
    int l = 0;
    while (true) {
      MGLevel<T>& L = mg.lv[l];
      L.g = make_grid(g.dim, n);
      long long f = L.g.field;
      L.x[0] = alloc<T>(f);
      L.x[1] = alloc<T>(f);
      L.b = alloc<T>(f);
      L.r = alloc<T>(f);
      L.jinv = alloc<T>(f);
      L.m = l == 0 ? nullptr : alloc<T>(f);
      mg.cur[l] = 0;
      ++l;
      if (n == 3) break;
      n = (n - 1) / 2 + 1;
    }
    mg.nlev = l;
  }

  void create(const ipm_grid* grid, const ipm_pde* p, double a, double b, const ipm_bounds* bd) {
    if (!grid || !bd) throw IpmError{IPM_EINVAL, "null grid or bounds"};
    int dim = grid->dim;
    if (dim != 2 && dim != 3) throw IpmError{IPM_EINVAL, "dim must be 2 or 3"};
    int n = grid->n[0];
    for (int k = 1; k < dim; ++k)
      if (grid->n[k] != n) throw IpmError{IPM_EINVAL, "grids must have equal node counts per direction"};
    if (n < 3 || ((n - 1) & (n - 2)) != 0)
      throw IpmError{IPM_EINVAL, "nodes per direction must be 2^k + 1 (k >= 1)"};
    if (!(a > 0.0) || !(b >= 0.0) || !std::isfinite(a) || !std::isfinite(b))
      throw IpmError{IPM_EINVAL, "need alpha > 0 and beta >= 0"};
    pde = p ? *p : ipm_pde{IPM_POISSON, 1.0, 0, 0.0};
    if (pde.kind != IPM_POISSON && pde.kind != IPM_CONVDIFF_SUPG && pde.kind != IPM_HEAT)
      throw IpmError{IPM_EINVAL, "unknown state equation"};
    if (pde.kind == IPM_CONVDIFF_SUPG && (dim != 2 || !(pde.eps > 0.0) || pde.wind != 0))
      throw IpmError{IPM_EINVAL, "convection-diffusion needs dim 2, eps > 0 and wind 0"};
    if (pde.kind == IPM_HEAT && (dim != 2 || n < 5 || n > 65 || !(pde.T > 0.0) ||
                                 !std::isfinite(pde.T)))
      throw IpmError{IPM_EINVAL, "heat equation needs dim 2, 5 <= n <= 65 and T > 0"};
    g = pde.kind == IPM_HEAT ? make_heat_grid(n, pde.T / (n - 2)) : make_grid(dim, n);
    alpha = a;
    beta = b;
    CK(cudaStreamCreateWithFlags(&own, cudaStreamNonBlocking));
    stream = own;
    CK(cudaMallocHost(&hbuf, sizeof(double) * 1024));
    long long f = F();
    st.y = alloc<double>(f);
    st.w = alloc<double>(f);
    st.v = alloc<double>(f);
    st.p = alloc<double>(f);
    st.lya = alloc<double>(f);
    st.lyb = alloc<double>(f);
    st.lwa = alloc<double>(f);
    st.lwb = alloc<double>(f);
    st.lva = alloc<double>(f);
    st.lvb = alloc<double>(f);
    ya = alloc<double>(f);
    yb = alloc<double>(f);
    zbw = alloc<double>(f);
    zbv = alloc<double>(f);
    cy = alloc<double>(f);
    fvec = alloc<double>(f);
    glift = alloc<double>(f);
    ydbuf = alloc<double>(f);
    fbuf = alloc<double>(f);
    dg.thy = alloc<double>(f);
    dg.thw = alloc<double>(f);
    dg.thv = alloc<double>(f);
    dg.mh = alloc<double>(f);
    dg.thy32 = alloc<float>(f);
    dg.mh32 = alloc<float>(f);
    dg.thw32 = alloc<float>(f);
    dg.thv32 = alloc<float>(f);
    dg.thyff = alloc<float>(2 * f);
    zf32 = alloc<float>(3 * f);
    for (int q = 0; q < 3; ++q) pff[q] = alloc<float>(2 * f);
    rhs = alloc<double>(4 * f);
    dx = alloc<double>(4 * f);
    ktmp = alloc<double>(4 * f);
    for (int i = 0; i < 4; ++i) cheb64[i] = alloc<double>(f);
    for (int i = 0; i < 4; ++i) cheb32[i] = alloc<float>(f);
    build_mg(mg64);
    build_mg(mg32);
    if (pde.kind == IPM_CONVDIFF_SUPG) build_cd_operators();
    mgb64 = alloc<double>(f);
    mgx64[0] = alloc<double>(f);
    mgx64[1] = alloc<double>(f);
    mgb3 = alloc<float>(2 * f);
    mgxf[0] = alloc<float>(2 * f);
    mgxf[1] = alloc<float>(2 * f);
    mgm3 = alloc<float>(2 * f);
    part_rows = std::max<long long>(interior_blocks(g), 8 * kRedBlocks);
    part = alloc<double>(part_rows * 8);
    dout = alloc<double>(64);
    sc = alloc<double>(16);
    kdev = alloc<double>(4 * (kMaxRestart + 2));
    kff = alloc<float>(2 * 4 * (kMaxRestart + 2));
    dense = alloc<double>(nn());
    if (heat()) build_heat_mg();
    set_bounds(bd);
  }

  // ------------------------------------------------------------------------
  // Heat equation (Section 3.4), space-time layout: the hierarchy of one time level for
  // the level-by-level solves with M + tau K + diag(M_hat_k) in the Schur approximation.
  // ------------------------------------------------------------------------
  struct HeatMG {
    int nl = 0;
    GridDesc lg[kMaxCoarse];
    float* m[kMaxCoarse] = {};  // diag(M_hat) of every time level on each 2D level
    float* b32 = nullptr;       // right-hand side and iterate of the level being solved
    float* x32 = nullptr;
  } hmg;
  bool heat() const { return g.heat != 0; }

  void build_heat_mg() {
    int n = g.n, l = 0;
    while (true) {
      if (l >= kMaxCoarse) throw IpmError{IPM_EINVAL, "heat: too many levels"};
      hmg.lg[l] = make_grid(2, n);
      // level 0 reads the FP32 copy of M_hat of all time levels in place (plane stride
      // g.plane = field of the 2D grid); coarser levels hold n time levels each
      hmg.m[l] = l == 0 ? dg.mh32 : alloc<float>((long long)g.n * hmg.lg[l].field);
      ++l;
      if (n == 3) break;
      n = (n - 1) / 2 + 1;
    }
    hmg.nl = l;
    hmg.b32 = alloc<float>(F());
    hmg.x32 = alloc<float>(F());
  }

  // per IPM step: M_hat restricted to the coarser 2D levels of every time level
  void heat_setup() {
    for (int k = 1; k <= g.n - 2; ++k)
      for (int l = 1; l < hmg.nl; ++l)
        launch_mg_restrict<float>(hmg.lg[l - 1], hmg.lg[l], hmg.m[l - 1] + k * hmg.lg[l - 1].field,
                                  hmg.m[l] + k * hmg.lg[l].field, stream);
  }

  // x = (calL + M_hat)^{-1} t (forward in time) or (calL + M_hat)^{-T} t (backward): per time
  // level a 2D solve with M + tau K + diag(M_hat_k), `vcycles` FP32 V-cycles of the one-CTA
  // kernel, for the right-hand side t_k + M x_{k -+ 1}
  void heat_lm_solve(const double* t, double* x, bool transpose, const ipm_options& o) {
    const int nt = g.n - 2;
    MGCoarse<float> cl;
    cl.nl = hmg.nl;
    cl.general = 1;
    for (int l = 0; l < hmg.nl; ++l) {
      const double H = hmg.lg[l].h;
      cl.n[l] = hmg.lg[l].n;
      cl.pitch[l] = hmg.lg[l].pitch;
      // M + tau K on level l (Galerkin-consistent rediscretisation: the Q1 stiffness does
      // not scale with the mesh in 2D, the mass scales with H^2)
      cl.c0[l] = (float)(16.0 * H * H / 36.0 + 8.0 * g.tau / 3.0);
      cl.ce[l] = (float)(4.0 * H * H / 36.0 - g.tau / 3.0);
      cl.cc[l] = (float)(H * H / 36.0 - g.tau / 3.0);
    }
    const int cycles = std::max(1, o.vcycles);
    int k = 0;
    for (int step = 0; step < nt; ++step) {
      k = transpose ? nt - step : 1 + step;
      const int kp = step == 0 ? -1 : (transpose ? k + 1 : k - 1);
      launch_heat_plane_rhs(g, t, k, kp, hmg.x32, x, hmg.b32, stream);
      for (int l = 0; l < hmg.nl; ++l) cl.m[l] = hmg.m[l] + k * hmg.lg[l].field;
      for (int c = 0; c < cycles; ++c)
        launch_mg2_coarse<float>(cl, hmg.b32 + k * g.plane, hmg.x32 + k * g.plane, 0.8,
                                 o.smooth_pre, o.smooth_post, c > 0 ? 1 : 0, stream);
    }
    launch_heat_plane_store(g, k, hmg.x32, x, stream);
  }

  // ------------------------------------------------------------------------
  // Partial observation (the subsection on partial observations): the tracking term
  // integrates over the elements whose centre lies strictly inside a box; the state row
  // then carries M_s, which is singular, and GMRES is preconditioned with P_Pi.
  // ------------------------------------------------------------------------
  float* obs_dev = nullptr;
  double *pim_l = nullptr, *pim_r = nullptr, *zero64 = nullptr;

  void set_observation(const double* lo, const double* hi) {
    if (heat()) throw IpmError{IPM_EINVAL, "partial observation is not defined for the heat equation"};
    drop_graphs();  // captured launches carry the grid descriptor
    has_data = false;
    solved = false;
    if (!lo || !hi) {
      g.obs = nullptr;
      return;
    }
    if (!obs_dev) {
      obs_dev = alloc<float>(F());
      pim_l = alloc<double>(F());
      pim_r = alloc<double>(F());
      zero64 = alloc<double>(F());
    }
    const int n = g.n, ne = n - 1;
    std::vector<float> mask((size_t)F(), 0.f);
    long long observed = 0;
    for (int ez = 0; ez < (g.dim == 3 ? ne : 1); ++ez)
      for (int ey = 0; ey < ne; ++ey)
        for (int ex = 0; ex < ne; ++ex) {
          const double cx = (ex + 0.5) * g.h, cyy = (ey + 0.5) * g.h, cz = (ez + 0.5) * g.h;
          bool in = cx > lo[0] && cx < hi[0] && cyy > lo[1] && cyy < hi[1];
          if (g.dim == 3) in = in && cz > lo[2] && cz < hi[2];
          if (in) {
            mask[(size_t)node_index(g, ex, ey, g.dim == 3 ? ez : 0)] = 1.f;
            ++observed;
          }
        }
    if (observed == 0) throw IpmError{IPM_EINVAL, "the observation box contains no element"};
    CK(cudaMemcpyAsync(obs_dev, mask.data(), sizeof(float) * mask.size(), cudaMemcpyHostToDevice,
                       stream));
    sync();  // the host mask goes out of scope
    g.obs = obs_dev;
  }

  // z = P_Pi^{-1} r: the permuted block-triangular preconditioner applied by three solves,
  // v2 = Z^{-1} r_z, v1 = L^{-1} (M_bar v2 + r_p), v3 = S_Pi_hat^{-1} ((M_s + Theta_y) v1 - r_y),
  // S_Pi_hat^{-1} = (L + M_r)^{-1} L (L^T + M_l)^{-1}; every inverse by V-cycles (M_l, M_r
  // lumped to diagonals for the smoother's operator)
  void precond_pi(const double* r, double* z, const ipm_options& o) {
    const long long f = F();
    int p2 = ph_begin(2);
    launch_zblock(g, alpha * mass_diag(g), r + f, r + 2 * f, dg.thw, dg.thv, z + f, z + 2 * f,
                  stream);
    // t = -(M z_w - M z_v + r_p)
    launch_coupling<double>(g, opL(), zero64, z + f, z + 2 * f, r + 3 * f, 1, mg64.lv[0].b, stream);
    ph_end(p2);
    int p3 = ph_begin(3);
    mg_setup(mg64, zero64);
    const double* x1 = mg_solve(mg64, 0, o);
    launch_axpby(z, x1, -1.0, 0.0, f, stream);  // v1 = -L^{-1} t
    mg_setup(mg64, pim_l);
    launch_track_theta_minus(g, z, dg.thy, r, mg64.lv[0].b, stream);
    const double* a1 = mg_solve(mg64, 1, o);
    launch_coupling<double>(g, opL(), a1, zero64, zero64, zero64, 1, mg64.lv[0].b, stream);
    mg_setup(mg64, pim_r);
    const double* c1 = mg_solve(mg64, 0, o);
    launch_convert<double, double>(g, c1, z + 3 * f, stream);
    ph_end(p3);
  }

  // P^{-1} r for the heat equation (P_T of Section 4 with the time-dependent Schur
  // approximation of Section 3.4): Chebyshev for tau calM + Theta_y, the pointwise z-block
  // with tau D_M, the coupling with calL, and the level-by-level solves with calL + M_hat
  void precond_heat(const double* r, double* z, int tri, const ipm_options& o) {
    const long long f = F();
    const bool mixed_cheb = o.precision == IPM_PREC_MIXED && !(o.kernel_flags & 4);
    int p1 = ph_begin(1);
    if (mixed_cheb) cheb_apply<float, double>(r, dg.thy32, z, o.cheb_steps, cheb32);
    else cheb_apply<double, double>(r, dg.thy, z, o.cheb_steps, cheb64);
    ph_end(p1);
    int p2 = ph_begin(2);
    launch_zblock(g, alpha * mass_diag(g), r + f, r + 2 * f, dg.thw, dg.thv, z + f, z + 2 * f,
                  stream);
    double* t = mg64.lv[0].b;
    double* s1 = mg64.lv[0].r;
    launch_coupling<double>(g, opL(), z, z + f, z + 2 * f, r + 3 * f, tri, t, stream);
    ph_end(p2);
    int p3 = ph_begin(3);
    heat_lm_solve(t, s1, false, o);
    ph_end(p3);
    int p4 = ph_begin(4);
    launch_mass_theta<double>(g, s1, dg.thy, t, stream);
    ph_end(p4);
    int p5 = ph_begin(3);
    heat_lm_solve(t, z + 3 * f, true, o);
    ph_end(p5);
  }

  // convection-diffusion: the SUPG operator rediscretised on every multigrid level, each
  // with its own element Peclet numbers. (Galerkin P^T L P operators keep the fine grid's
  // SUPG parameter and are under-stabilised on coarse grids, where damped Jacobi diverges.)
  void build_cd_operators() {
    lvop.resize(mg64.nlev);
    for (int l = 0; l < mg64.nlev; ++l) {
      const GridDesc& gl = mg64.lv[l].g;
      double* c64 = alloc<double>(9 * gl.field);
      float* c32 = alloc<float>(9 * gl.field);
      launch_cd_coef(gl, pde.eps, c64, stream);
      launch_to_float(9 * gl.field, c64, c32, stream);
      lvop[l] = OpL{c64, c32};
    }
    sync();
  }

  // reuse the solver (same grid and state equation) for a new problem
  void reset(double a, double b, const ipm_bounds* bd) {
    if (!bd) throw IpmError{IPM_EINVAL, "null bounds"};
    if (!(a > 0.0) || !(b >= 0.0) || !std::isfinite(a) || !std::isfinite(b))
      throw IpmError{IPM_EINVAL, "need alpha > 0 and beta >= 0"};
    set_bounds(bd);
    alpha = a;
    beta = b;
    drop_graphs();  // captured kernels carry alpha-dependent arguments
    has_data = false;
    solved = false;
  }

  // bounds -> fields ya, yb, zbw = max(u_b, 0) = u_b, zbv = -min(u_a, 0) = -u_a
  void set_bounds(const ipm_bounds* bd) {
    long long m = nn();
    std::vector<double> ua(m), ub(m), yav(m), ybv(m);
    for (long long t = 0; t < m; ++t) {
      ua[t] = bd->ua_v ? bd->ua_v[t] : bd->ua;
      ub[t] = bd->ub_v ? bd->ub_v[t] : bd->ub;
      yav[t] = bd->ya_v ? bd->ya_v[t] : bd->ya;
      ybv[t] = bd->yb_v ? bd->yb_v[t] : bd->yb;
    }
    // validate interior entries
    int n = g.n;
    for (long long t = 0; t < m; ++t) {
      int i = (int)(t % n), j = (int)((t / n) % n), k = g.dim == 3 ? (int)(t / ((long long)n * n)) : 1;
      bool bnd = i == 0 || j == 0 || i == n - 1 || j == n - 1 || (g.dim == 3 && (k == 0 || k == n - 1));
      if (bnd) continue;
      if (!(ua[t] < 0.0) || !(ub[t] > 0.0) || std::isnan(ua[t]) || std::isnan(ub[t]))
        throw IpmError{IPM_EINVAL, "control bounds must satisfy u_a < 0 < u_b"};
      if (std::isnan(yav[t]) || std::isnan(ybv[t]) || !(yav[t] < ybv[t]))
        throw IpmError{IPM_EINVAL, "state bounds must satisfy y_a < y_b"};
      if (yav[t] == INFINITY || ybv[t] == -INFINITY)
        throw IpmError{IPM_EINVAL, "state bounds are infeasible"};
      if (heat() && (std::isfinite(yav[t]) || std::isfinite(ybv[t])))
        throw IpmError{IPM_EINVAL, "the heat equation takes control bounds only"};
    }
    for (long long t = 0; t < m; ++t) {
      ub[t] = std::max(ub[t], 0.0);
      ua[t] = -std::min(ua[t], 0.0);
    }
    upload_field(ybv.data(), yb, 1);
    upload_field(yav.data(), ya, 1);
    upload_field(ub.data(), zbw, 1);
    upload_field(ua.data(), zbv, 1);
    sync();
  }

  void upload_field(const double* host, double* field, int mode) {
    CK(cudaMemcpyAsync(dense, host, sizeof(double) * nn(), cudaMemcpyHostToDevice, stream));
    launch_pack(g, dense, field, mode, stream);
  }

  void set_data(const double* yd, const double* f, const double* gb, bool device) {
    // pack y_d and f with their boundary values into their own buffers (never into
    // Krylov vectors, whose boundary entries must stay zero), g -> glift (boundary only)
    double* ydp = ydbuf;
    double* fp = fbuf;
    auto put = [&](const double* src, double* dst, int mode) {
      if (!src) {
        launch_pack(g, nullptr, dst, mode, stream);
        return;
      }
      if (device) {
        launch_pack(g, src, dst, mode, stream);
      } else {
        CK(cudaMemcpyAsync(dense, src, sizeof(double) * nn(), cudaMemcpyHostToDevice, stream));
        launch_pack(g, dense, dst, mode, stream);
      }
    };
    put(yd, ydp, 0);
    put(f, fp, 0);
    put(gb, glift, 2);
    launch_setup_data(g, ydp, fp, glift, opL(), cy, fvec, stream);
    launch_element_mass_form(g, ydp, glift, part, dout, stream);
    launch_setup_norms(g, cy, fvec, bounds(), part, dout + 1, stream);
    fetch(dout, 4);
    c0 = hbuf[0];
    ncy = std::sqrt(hbuf[1]);
    nf = std::sqrt(hbuf[2]);
    nbounds = hbuf[3];
    nd = lumped_mass(g) * std::sqrt((double)nI());
    has_data = true;
    solved = false;
  }

  // ------------------------------------------------------------------------
  // Multigrid V-cycles on L + diag(m)
  // ------------------------------------------------------------------------
  template <typename T>
  void mg_setup(MGHier<T>& mg, T* m0) {
    mg.lv[0].m = m0;
    for (int l = 1; l < mg.nlev; ++l)
      launch_mg_restrict<T>(mg.lv[l - 1].g, mg.lv[l].g, mg.lv[l - 1].m, mg.lv[l].m, stream);
    for (int l = 0; l < mg.nlev; ++l)
      launch_mg_jinv<T>(mg.lv[l].g, opl(l), mg.lv[l].m, omega(), mg.lv[l].jinv, stream);
  }

  template <typename T>
  void vcycle(MGHier<T>& mg, int l, bool zero_x, int tr, const ipm_options& o) {
    MGLevel<T>& L = mg.lv[l];
    int& cur = mg.cur[l];
    if (l == mg.nlev - 1) {
      launch_mg_coarsest<T>(L.g, opl(l), L.b, L.m, L.x[cur], stream);
      return;
    }
    bool z = zero_x;
    for (int i = 0; i < o.smooth_pre; ++i) {
      int pr = (l == 0 && !z) ? prof_begin_kind(0, 0) : -1;
      launch_mg_smooth<T>(L.g, opl(l), L.x[cur], L.x[1 - cur], L.b, L.m, L.jinv, z, tr, stream);
      prof_end(pr);
      cur = 1 - cur;
      z = false;
    }
    if (z) launch_mg_zero<T>(L.g, L.x[cur], stream);
    launch_mg_residual<T>(L.g, opl(l), L.x[cur], L.b, L.m, L.r, tr, stream);
    MGLevel<T>& C = mg.lv[l + 1];
    launch_mg_restrict<T>(L.g, C.g, L.r, C.b, stream);
    vcycle(mg, l + 1, true, tr, o);
    launch_mg_prolong_add<T>(L.g, C.g, C.x[mg.cur[l + 1]], L.x[cur], stream);
    for (int i = 0; i < o.smooth_post; ++i) {
      int pr = l == 0 ? prof_begin_kind(1, 14) : -1;
      launch_mg_smooth<T>(L.g, opl(l), L.x[cur], L.x[1 - cur], L.b, L.m, L.jinv, 0, tr, stream);
      prof_end(pr);
      cur = 1 - cur;
    }
  }

  // first level handled by the one-CTA coarse kernel (2D Poisson fused path)
  template <typename T>
  int coarse_start(const MGHier<T>& mg) const {
    // FP32: levels up to 65^2 in one CTA. FP64 runs at 1/64 of the FP32 rate on this
    // GPU, so one SM is slow: only the last three levels go into the one-CTA kernel.
    const int limit = sizeof(T) == 4 ? 65 : 9;
    for (int l = 0; l < mg.nlev; ++l)
      if (mg.lv[l].g.n <= limit) return l;
    return mg.nlev - 1;
  }
  bool fused_mg() const { return g.dim == 2 && fused && nu_fits && lvop.empty(); }
  bool nu_fits = true;  // fused tiles hold up to 8 sweeps of halo

  // levels below the finest one in one persistent cooperative launch (FP32, 5 + 5 sweeps):
  // levels above 33^2 as tiles, the rest in one CTA; returns false when not applicable
  bool use_mid_cycle = false;  // kernel_flags bit 7 sets it
  GridBarrier* gbar = nullptr;
  int mid_blocks = -1;  // blocks of the cooperative launch (0: not available)
#ifndef IPM_MID_TOP
#define IPM_MID_TOP 129
#endif
  // levels [lt, nlev) of the mixed FP32 hierarchy in one persistent launch: levels above
  // 33^2 (and at most IPM_MID_TOP per direction) as tiles, the rest in one CTA; the levels
  // [0, lt) above keep one launch per level. Returns lt, or 0 when not applicable.
  int prepare_mid(MGHier<float>& mg, const ipm_options& o, MidCycle& mc) {
    if (!use_mid_cycle || o.smooth_pre != 5 || o.smooth_post != 5) return 0;
    int lt = 1;
    while (lt < mg.nlev && mg.lv[lt].g.n > IPM_MID_TOP) ++lt;
    int lm = lt;
    while (lm < mg.nlev && mg.lv[lm].g.n > 33) ++lm;
    const int nt = lm - lt;  // tiled levels in the persistent launch
    if (nt < 1 || nt > kMaxMid || mg.nlev - lm > kMaxCoarse) return 0;
    mc.nt = nt;
    for (int t = 0; t < nt; ++t) {
      MGLevel<float>& L = mg.lv[lt + t];
      mc.g[t] = L.g;
      mc.xa[t] = L.x[mg.cur[lt + t]];
      mc.xb[t] = L.x[1 - mg.cur[lt + t]];
      mc.b[t] = L.b;
      mc.m[t] = L.m;
      mc.bnext[t] = mg.lv[lt + t + 1].b;
    }
    mc.g[nt] = mg.lv[lm].g;
    mc.cl.nl = mg.nlev - lm;
    mc.cl.general = 0;
    for (int l = lm; l < mg.nlev; ++l) {
      mc.cl.n[l - lm] = mg.lv[l].g.n;
      mc.cl.pitch[l - lm] = mg.lv[l].g.pitch;
      mc.cl.m[l - lm] = mg.lv[l].m;
    }
    mc.xcoarse = mg.lv[lm].x[mg.cur[lm]];
    if (mid_blocks < 0) mid_blocks = mg2_mid_blocks(mc);
    if (mid_blocks <= 0) return 0;
    if (!gbar) gbar = alloc<GridBarrier>(1);
    return lt;
  }

  // one V-cycle with the fused kernels (same operator, smoother and transfers)
  template <typename T>
  void vcycle_fused(MGHier<T>& mg, bool zero_x, const ipm_options& o) {
    if constexpr (std::is_same<T, float>::value) {
      // the upper levels as their own launches, everything from IPM_MID_TOP down in one
      // persistent launch
      MidCycle mc;
      const int lt = prepare_mid(mg, o, mc);
      if (lt > 0) {
        for (int l = 0; l < lt; ++l) {
          MGLevel<float>& L = mg.lv[l];
          int& cur = mg.cur[l];
          const bool z = l > 0 || zero_x;
          int pr = prof_begin_kind(l == 0 ? 0 : 4, l == 0 && zero_x ? 13 : 0,
                                   pre_pass(L.g.n, o.smooth_pre, z), pre_once(L.g.n, z));
          int ph = ph_begin(l == 0 ? 9 : 11);
          launch_mg2_pre_restrict<float>(L.g, mg.lv[l + 1].g, L.x[cur], L.x[1 - cur], L.b, L.m,
                                         mg.lv[l + 1].b, omega(), o.smooth_pre, z ? 1 : 0,
                                         stream);
          ph_end(ph);
          prof_end(pr);
          cur = 1 - cur;
        }
        double mbp = 0.0, mbo = 0.0;
        for (int l = lt; l + 1 < mg.nlev; ++l) {
          mbp += pre_pass(mg.lv[l].g.n, 5, true) + post_pass(mg.lv[l].g.n, 5);
          mbo += pre_once(mg.lv[l].g.n, true) + post_once(mg.lv[l].g.n);
        }
        int pr2 = prof_begin_kind(2, 15, mbp, mbo);
        int ph2 = ph_begin(12);
        launch_mg2_mid_cycle(mc, gbar, omega(), mid_blocks, stream);
        ph_end(ph2);
        prof_end(pr2);
        for (int l = lt - 1; l >= 0; --l) {
          MGLevel<float>& L = mg.lv[l];
          int& cur = mg.cur[l];
          int pr3 = prof_begin_kind(l == 0 ? 1 : 4, 14, post_pass(L.g.n, 5), post_once(L.g.n));
          int ph3 = ph_begin(l == 0 ? 10 : 11);
          launch_mg2_prolong_post<float>(L.g, mg.lv[l + 1].g, L.x[cur], mg.lv[l + 1].x[mg.cur[l + 1]],
                                         L.x[1 - cur], L.b, L.m, omega(), o.smooth_post, stream);
          ph_end(ph3);
          prof_end(pr3);
          cur = 1 - cur;
        }
        return;
      }
    }
    const int lc = coarse_start(mg);
    for (int l = 0; l < lc; ++l) {
      MGLevel<T>& L = mg.lv[l];
      int& cur = mg.cur[l];
      const bool z = l > 0 || zero_x;
      const int n = L.g.n;
      int pr = prof_begin_kind(l == 0 ? 0 : 4, l == 0 && zero_x ? 13 : 0,
                               pre_pass(n, o.smooth_pre, z), pre_once(n, z));
      int ph = ph_begin(l == 0 ? 9 : 11);
      launch_mg2_pre_restrict<T>(L.g, mg.lv[l + 1].g, L.x[cur], L.x[1 - cur], L.b, L.m,
                                 mg.lv[l + 1].b, omega(), o.smooth_pre, z ? 1 : 0, stream);
      ph_end(ph);
      prof_end(pr);
      cur = 1 - cur;
    }
    MGCoarse<T> cl;
    cl.general = 0;
    cl.nl = mg.nlev - lc;
    for (int l = lc; l < mg.nlev; ++l) {
      cl.n[l - lc] = mg.lv[l].g.n;
      cl.pitch[l - lc] = mg.lv[l].g.pitch;
      cl.m[l - lc] = mg.lv[l].m;
    }
    // the one-CTA cycle starts from zero below the top level; when it is the top
    // level itself it continues from the current iterate after the first cycle
    double cbp = 0.0, cbo = 0.0;
    for (int l = lc; l + 1 < mg.nlev; ++l) {
      cbp += pre_pass(mg.lv[l].g.n, o.smooth_pre, true) + post_pass(mg.lv[l].g.n, o.smooth_post);
      cbo += u2(mg.lv[l].g.n) * 4 * (l == lc ? 3.0 : 1.0);  // b, x of the top; m of every level
    }
    int prc = prof_begin_kind(2, 15, cbp, cbo);
    int phc = ph_begin(12);
    launch_mg2_coarse<T>(cl, mg.lv[lc].b, mg.lv[lc].x[mg.cur[lc]], omega(), o.smooth_pre,
                         o.smooth_post, (lc == 0 && !zero_x) ? 1 : 0, stream);
    ph_end(phc);
    prof_end(prc);
    for (int l = lc - 1; l >= 0; --l) {
      MGLevel<T>& L = mg.lv[l];
      int& cur = mg.cur[l];
      int pr = prof_begin_kind(l == 0 ? 1 : 4, 14, post_pass(L.g.n, o.smooth_post),
                               post_once(L.g.n));
      int ph = ph_begin(l == 0 ? 10 : 11);
      launch_mg2_prolong_post<T>(L.g, mg.lv[l + 1].g, L.x[cur], mg.lv[l + 1].x[mg.cur[l + 1]],
                                 L.x[1 - cur], L.b, L.m, omega(), o.smooth_post, stream);
      ph_end(ph);
      prof_end(pr);
      cur = 1 - cur;
    }
  }

  // Mixed-precision multigrid solve of (L + M_hat) x = b64 (FP64 right-hand side):
  // the cycle iterate and its residual stay in FP64 on the finest level, every V-cycle
  // runs in FP32 on the correction equation from zero: x_{k+1} = x_k + V(b - A x_k),
  // the same operator as `vcycles` cycles from zero. In FP32 alone the finest-level
  // residual of a smooth iterate loses its digits to cancellation in the stiffness
  // stencil (8 x_c - neighbours ~ h^2 x''), which slows the outer Krylov method.
  // float-float outer residual: 2D Poisson (constant-coefficient stencil) only
  bool use_ff_outer() const { return ff_outer && g.dim == 2 && lvop.empty(); }

  // FP32 multigrid setup of the mixed path from dg.mh (and its FP32 copy dg.mh32)
  void mg_setup_mixed() {
    mg_setup(mg32, dg.mh32);
    if (use_ff_outer()) launch_split3_ff(g, dg.mh, mgm3, mgm3 + F(), stream);
    if (autotune && fused_mg()) autotune_tiles();
  }

  // tile shapes of the FP32 tiled levels: timed once per grid size and device in this
  // process (kernel_flags bit 9 keeps the fixed shapes). Runs eagerly, before any capture,
  // on this solver's level buffers, which the following cycle overwrites.
  bool autotune = true;
  bool ff_operator = true;  // mixed FGMRES: saddle operator in float-float (kernel_flags bit 10)
  void autotune_tiles() {
    const int lc = coarse_start(mg32);
    for (int l = 0; l < lc; ++l) {
      MGLevel<float>& L = mg32.lv[l];
      if (mg2_is_tuned(L.g.n)) continue;
      MGLevel<float>& C = mg32.lv[l + 1];
      if (mg2_autotune(L.g, C.g, L.x[0], L.x[1], L.b, L.m, C.b, C.x[0], omega(), stream) != 0)
        throw IpmError{IPM_ECUDA, "tile autotuning failed"};
    }
  }

  // float-float outer iterate (high part, then low part); right-hand side as FP64 (b64) or
  // float-float planes (bff), result to FP64 (out) or float-float planes (outff)
  void mg_solve_mixed_ff(const double* b64, const float* bff, double* out, float* outff, int tr,
                         const ipm_options& o) {
    MGLevel<float>& L0 = mg32.lv[0];
    const int cycles = std::max(1, o.vcycles);
    const long long f = F();
    if (bff) CK(cudaMemcpyAsync(L0.b, bff, sizeof(float) * f, cudaMemcpyDeviceToDevice, stream));
    else launch_convert<double, float>(g, b64, L0.b, stream);
    for (int c = 0; c < cycles; ++c) {
      if (fused_mg()) vcycle_fused(mg32, true, o);
      else vcycle(mg32, 0, true, tr, o);
      const float* e = L0.x[mg32.cur[0]];
      const bool last = c == cycles - 1;
      float* xin = mgxf[(c + 1) & 1];
      float* xout = mgxf[c & 1];
      launch_mg_outer_ff(g, xin, xin + f, e, b64, bff, mgb3, mgb3 + f, mgm3, mgm3 + f, xout,
                         xout + f, last ? nullptr : L0.b, last ? out : nullptr,
                         last ? outff : nullptr, c == 0 ? 1 : 0, stream);
    }
  }

  void mg_solve_mixed(const double* b64, double* out, int tr, const ipm_options& o) {
    if (use_ff_outer()) {
      mg_solve_mixed_ff(b64, nullptr, out, nullptr, tr, o);
      return;
    }
    MGLevel<float>& L0 = mg32.lv[0];
    const int cycles = std::max(1, o.vcycles);
    launch_convert<double, float>(g, b64, L0.b, stream);
    const double* xprev = nullptr;
    int xb = 0;
    for (int c = 0; c < cycles; ++c) {
      float* e;
      if (fused_mg()) {
        vcycle_fused(mg32, true, o);
      } else {
        vcycle(mg32, 0, true, tr, o);
      }
      e = L0.x[mg32.cur[0]];
      const bool last = c == cycles - 1;
      double* xnew = last ? out : mgx64[xb];
      launch_mg_outer(g, opL(), xprev, e, b64, dg.mh, xnew, last ? nullptr : L0.b, tr, stream);
      xprev = xnew;
      xb ^= 1;
    }
  }

  // x = (vcycles V-cycles from zero) applied to lv[0].b; returns the level-0 iterate
  template <typename T>
  T* mg_solve(MGHier<T>& mg, int tr, const ipm_options& o) {
    for (int c = 0; c < std::max(1, o.vcycles); ++c) {
      if (fused_mg()) vcycle_fused(mg, c == 0, o);  // L symmetric: tr needs no change
      else vcycle(mg, 0, c == 0, tr, o);
    }
    return mg.lv[0].x[mg.cur[0]];
  }

  // ------------------------------------------------------------------------
  // Chebyshev semi-iteration for (M + Theta_y) x = r_y (Section 4.1)
  // ------------------------------------------------------------------------
  // 2D: blocks of up to 5 steps per launch (temporal blocking), same recurrence
  template <typename T>
  void cheb_apply_fused(const double* r, const T* thy, double* z, int steps, T* const* buf) {
    const double lmin = 0.25, lmax = 2.25;
    double theta = 0.5 * (lmax + lmin), delta = 0.5 * (lmax - lmin), sig = theta / delta;
    std::vector<double> om(steps + 1, 0.0);
    double rho = 1.0 / sig;
    for (int k = 1; k < steps; ++k) {
      double rho_new = 1.0 / (2.0 * sig - rho);
      om[k] = 2.0 * sig * rho_new;
      rho = rho_new;
    }
    ChebSteps cs;
    cs.gamma = 1.0 / theta;
    cs.dM = mass_diag(g);
    cs.mscale = g.h * g.h / 36.0;
    int k = 1, pair = 0;
    bool first = true;
    while (true) {
      int ns = std::min(5, steps - k);
      cs.ns = ns;
      for (int q = 0; q < ns; ++q) cs.omega[q] = om[k + q];
      bool last = k + ns == steps;
      launch_cheb2_block<T, double, double>(g, cs, r, thy, buf[2 * pair], buf[2 * pair + 1],
                                            buf[2 * (1 - pair)], buf[2 * (1 - pair) + 1],
                                            last ? z : nullptr, first ? 1 : 0, stream);
      k += ns;
      first = false;
      pair = 1 - pair;
      if (last) break;
    }
  }

  template <typename T, typename To>
  void cheb_apply(const double* r, const T* thy, To* z, int steps, T* const* buf) {
    if (g.dim == 2 && fused) {
      cheb_apply_fused<T>(r, thy, (double*)z, steps, buf);
      return;
    }
    // Q1 element bounds of D_M^{-1} M; the heat layout's masses act within a 2D time level
    const bool d2 = g.dim == 2 || heat();
    double lmin = d2 ? 0.25 : 0.125, lmax = d2 ? 2.25 : 3.375;
    double theta = 0.5 * (lmax + lmin), delta = 0.5 * (lmax - lmin), sig = theta / delta;
    T* bT = buf[2];
    T* cur = buf[0];
    T* prev = buf[1];
    double dM = mass_diag(g);
    launch_cheb_init<T>(g, r, thy, dM, 1.0 / theta, bT, cur, prev, stream);
    double rho = 1.0 / sig;
    for (int k = 1; k < steps; ++k) {
      double rho_new = 1.0 / (2.0 * sig - rho);
      double om = 2.0 * sig * rho_new;
      rho = rho_new;
      if (k == steps - 1) {
        launch_cheb_step<T, To>(g, cur, prev, bT, thy, dM, om, 1.0 / theta, z, stream);
        return;
      }
      launch_cheb_step<T, T>(g, cur, prev, bT, thy, dM, om, 1.0 / theta, prev, stream);
      std::swap(cur, prev);
    }
    launch_convert<T, To>(g, cur, z, stream);  // steps <= 1
  }

  // z = P^{-1} r, P = P_T (tri) or P_D (Section 4.2)
  void precond(const double* r, double* z, int tri, const ipm_options& o) {
    if (heat()) {
      precond_heat(r, z, tri, o);
      return;
    }
    if (g.obs) {
      precond_pi(r, z, o);
      return;
    }
    long long f = F();
    // kernel_flags bits 2 / 3 keep the Chebyshev and z-block / multigrid stage in FP64 on
    // the mixed path
    bool mixed_cheb = o.precision == IPM_PREC_MIXED && !(o.kernel_flags & 4);
    bool mixed = o.precision == IPM_PREC_MIXED && !(o.kernel_flags & 8);
    int p1 = ph_begin(1);
    if (mixed_cheb) cheb_apply<float, double>(r, dg.thy32, z, o.cheb_steps, cheb32);
    else cheb_apply<double, double>(r, dg.thy, z, o.cheb_steps, cheb64);
    ph_end(p1);
    int p2 = ph_begin(2);
    if (mixed_cheb)
      launch_zblock32(g, alpha * mass_diag(g), r + f, r + 2 * f, dg.thw32, dg.thv32, z + f,
                      z + 2 * f, stream);
    else
      launch_zblock(g, alpha * mass_diag(g), r + f, r + 2 * f, dg.thw, dg.thv, z + f, z + 2 * f,
                    stream);
    if (mixed) launch_coupling<double>(g, opL(), z, z + f, z + 2 * f, r + 3 * f, tri, mgb64, stream);
    else launch_coupling<double>(g, opL(), z, z + f, z + 2 * f, r + 3 * f, tri, mg64.lv[0].b, stream);
    ph_end(p2);
    if (mixed) {
      // S_hat^{-1} t = (L + M_hat)^{-T} (M + Theta_y) (L + M_hat)^{-1} t, FP32 cycles with
      // float-float (2D Poisson) or FP64 outer residuals; s1 is kept in FP64 for the
      // (M + Theta_y) product
      double* s1 = mg64.lv[0].r;  // an FP64 field of the finest level, free during this solve
      int p3 = ph_begin(3);
      mg_solve_mixed(mgb64, s1, 0, o);
      ph_end(p3);
      int p4 = ph_begin(4);
      launch_mass_theta<double>(g, s1, dg.thy, mgb64, stream);
      ph_end(p4);
      int p5 = ph_begin(3);
      mg_solve_mixed(mgb64, z + 3 * f, 1, o);
      ph_end(p5);
    } else {
      int p3 = ph_begin(3);
      double* s1 = mg_solve(mg64, 0, o);
      ph_end(p3);
      int p4 = ph_begin(4);
      launch_mass_theta<double>(g, s1, dg.thy, mg64.lv[0].b, stream);
      ph_end(p4);
      int p5 = ph_begin(3);
      double* xp = mg_solve(mg64, 1, o);
      ph_end(p5);
      int p6 = ph_begin(4);
      launch_convert<double, double>(g, xp, z + 3 * f, stream);
      ph_end(p6);
    }
  }

  // P_T^{-1} v for a float-float Krylov vector v (2D Poisson, mixed precision): the y- and
  // z-blocks from the FP32 high parts, the coupling and the Schur stage in float-float, so
  // that no FP64 arithmetic runs but the conversion of z to FP64 for the FGMRES basis Z.
  bool precond_ff_ok(const ipm_options& o, int tri) const {
    const int k = o.cheb_steps - 1;  // Chebyshev blocks of 5 steps, the last of 4 or 5
    return tri && krylov_ff && use_ff_outer() && fused && fused_mg() && !(o.kernel_flags & 76) &&
           k > 0 && (k % 5 == 0 || k % 5 == 4);
  }

  void cheb_apply_f32(const float* r32, double* z, float* z32, int steps) {
    const double lmin = 0.25, lmax = 2.25;
    double theta = 0.5 * (lmax + lmin), delta = 0.5 * (lmax - lmin), sig = theta / delta;
    std::vector<double> om(steps + 1, 0.0);
    double rho = 1.0 / sig;
    for (int k = 1; k < steps; ++k) {
      double rho_new = 1.0 / (2.0 * sig - rho);
      om[k] = 2.0 * sig * rho_new;
      rho = rho_new;
    }
    ChebSteps cs;
    cs.gamma = 1.0 / theta;
    cs.dM = mass_diag(g);
    cs.mscale = g.h * g.h / 36.0;
    float* const* buf = cheb32;
    int k = 1, pair = 0;
    bool first = true;
    while (true) {
      int ns = std::min(5, steps - k);
      cs.ns = ns;
      for (int q = 0; q < ns; ++q) cs.omega[q] = om[k + q];
      bool last = k + ns == steps;
      if (!launch_cheb2_rb_f32(g, cs, r32, dg.thy32, buf[2 * pair], buf[2 * pair + 1],
                               buf[2 * (1 - pair)], buf[2 * (1 - pair) + 1], last ? z : nullptr,
                               last ? z32 : nullptr, first ? 1 : 0, stream))
        throw IpmError{IPM_EINVAL, "Chebyshev block size without an FP32-input kernel"};
      k += ns;
      first = false;
      pair = 1 - pair;
      if (last) break;
    }
  }

  void precond_ff(const float* v, double* z, const ipm_options& o) {
    const long long f = F(), len = 4 * f;
    const float* vh = v;
    const float* vl = v + len;
    int p1 = ph_begin(1);
    cheb_apply_f32(vh, z, zf32, o.cheb_steps);
    ph_end(p1);
    int p2 = ph_begin(2);
    launch_zblock32f(g, alpha * mass_diag(g), vh + f, vh + 2 * f, dg.thw32, dg.thv32, z + f,
                     z + 2 * f, zf32 + f, zf32 + 2 * f, stream);
    launch_coupling_ff(g, zf32, zf32 + f, zf32 + 2 * f, vh + 3 * f, vl + 3 * f, pff[0],
                       pff[0] + f, stream);
    ph_end(p2);
    int p3 = ph_begin(3);
    mg_solve_mixed_ff(nullptr, pff[0], nullptr, pff[1], 0, o);
    ph_end(p3);
    int p4 = ph_begin(4);
    launch_mass_theta_ff(g, pff[1], pff[1] + f, dg.thyff, dg.thyff + f, pff[2], pff[2] + f,
                         stream);
    ph_end(p4);
    int p5 = ph_begin(3);
    mg_solve_mixed_ff(nullptr, pff[2], z + 3 * f, nullptr, 1, o);
    ph_end(p5);
  }

  void setup_precond(const ipm_options& o) {
    if (heat()) {
      heat_setup();
      return;
    }
    if (g.obs) {
      launch_pi_diags(g, alpha * mass_diag(g), lumped_mass(g), dg.thy, dg.thw, dg.thv, pim_l,
                      pim_r, stream);
      return;
    }
    if (o.precision == IPM_PREC_MIXED && !(o.kernel_flags & 8)) mg_setup_mixed();
    else mg_setup(mg64, dg.mh);
  }

  void newton_apply(const double* x, double* y) {
    const double ob = 11.0 * 8.0 * (double)nI();  // 7 fields read, 4 written, FP64
    int pr = prof_begin_kind(3, 16, ob, ob);
    launch_newton_apply(g, problem(), dg, x, y, stream);
    prof_end(pr);
  }

  double norm(const double* x, long long len) {
    launch_dot(x, x, len, part, dout, stream);
    fetch(dout, 1);
    return std::sqrt(hbuf[0]);
  }

  void ensure_krylov(const ipm_options& o) {
    long long f4 = 4 * F();
    if (o.krylov == IPM_KRYLOV_GMRES_PT) {
      if (vcap < o.restart) {
        // buffers only grow; earlier ones stay owned by the arena
        V = alloc<double>((long long)(o.restart + 1) * f4);
        Z = alloc<double>((long long)o.restart * f4);
        vcap = o.restart;
        vlayout = -1;
      }
    } else if (!mr[0]) {
      for (int i = 0; i < 16; ++i) mr[i] = alloc<double>(f4);
    }
  }

  // One Arnoldi step j of FGMRES, enqueued on the stream (no host synchronisation):
  // normalise V_j by the squared norm left by step j-1, Z_j = P^{-1} V_j,
  // V_{j+1} = A Z_j, two classical Gram-Schmidt passes against V_0..V_j, the squared
  // norm of V_{j+1}, and a copy of the coefficients into the pinned host buffer.
  // Float-float form of the step: V_j and w in float-float (Gram-Schmidt and norms at FP32
  // instruction rates), Z_j and the operator in FP64; P^{-1} reads V_j converted to FP64.
  void arnoldi_body_ff(const ipm_options& o, int j, long long stride, long long len, int tri) {
    float* Vf = (float*)V;
    const long long sf = 2 * stride;  // floats per basis vector
    float* vj = Vf + (long long)j * sf;
    double* zj = Z + (long long)j * stride;
    float* w = Vf + (long long)(j + 1) * sf;
    const int K = kMaxRestart + 2;
    int p0 = ph_begin(5);
    if (j > 0) launch_scale_ff(vj, kff + 2 * (2 * K), len, stream);
    const bool pff_ok = precond_ff_ok(o, tri);
    if (!pff_ok) launch_from_ff(ktmp, vj, len, stream);
    ph_end(p0);
    if (pff_ok) precond_ff(vj, zj, o);
    else precond(ktmp, zj, tri, o);
    int p1 = ph_begin(6);
    const double ob = 11.0 * 8.0 * (double)nI();
    int pr = prof_begin_kind(3, 16, ob, ob);
    if (ff_operator && newton_apply_ff2_ok(g, problem()))
      launch_newton_apply_ff2(g, problem(), dg, zj, w, stream);
    else
      launch_newton_apply_ff(g, problem(), dg, zj, w, stream);
    prof_end(pr);
    ph_end(p1);
    int p2 = ph_begin(7);
    launch_multidot_ff(Vf, sf, j + 1, w, len, part, kdev, kff, 1, stream);
    ph_end(p2);
    int p3 = ph_begin(8);
    launch_axpy_multi_ff(w, Vf, sf, j + 1, kff, -1.0, len, stream);
    ph_end(p3);
    int p4 = ph_begin(7);
    launch_multidot_ff(Vf, sf, j + 1, w, len, part, kdev + K, kff + 2 * K, 0, stream);
    ph_end(p4);
    int p5 = ph_begin(8);
    launch_axpy_multi_ff(w, Vf, sf, j + 1, kff + 2 * K, -1.0, len, stream);
    ph_end(p5);
    int p6 = ph_begin(5);
    launch_norm2_ff(w, len, part, kdev + 2 * K, kff + 2 * (2 * K), stream);
    ph_end(p6);
    CK(cudaMemcpyAsync(hbuf, kdev, sizeof(double) * (2 * K + 1), cudaMemcpyDeviceToHost, stream));
  }

  void arnoldi_body(const ipm_options& o, int j, long long stride, long long len, int tri) {
    if (krylov_ff) {
      arnoldi_body_ff(o, j, stride, len, tri);
      return;
    }
    double* vj = V + (long long)j * stride;
    double* zj = Z + (long long)j * stride;
    double* w = V + (long long)(j + 1) * stride;
    const int K = kMaxRestart + 2;
    int p0 = ph_begin(5);
    if (j > 0) launch_scale_rsqrt(vj, vj, kdev + 2 * K, len, stream);
    ph_end(p0);
    precond(vj, zj, tri, o);
    int p1 = ph_begin(6);
    newton_apply(zj, w);
    ph_end(p1);
    int p2 = ph_begin(7);
    launch_multidot(V, stride, j + 1, w, len, part, kdev, stream);
    ph_end(p2);
    int p3 = ph_begin(8);
    launch_axpy_multi(w, V, stride, j + 1, kdev, -1.0, len, stream);
    ph_end(p3);
    int p4 = ph_begin(7);
    launch_multidot(V, stride, j + 1, w, len, part, kdev + K, stream);
    ph_end(p4);
    int p5 = ph_begin(8);
    launch_axpy_multi(w, V, stride, j + 1, kdev + K, -1.0, len, stream);
    ph_end(p5);
    int p6 = ph_begin(5);
    launch_dot(w, w, len, part, kdev + 2 * K, stream);
    ph_end(p6);
    CK(cudaMemcpyAsync(hbuf, kdev, sizeof(double) * (2 * K + 1), cudaMemcpyDeviceToHost, stream));
  }

  void arnoldi_step(const ipm_options& o, int j, long long stride, long long len, int tri) {
    long long key = ((long long)o.precision << 40) ^ ((long long)tri << 39) ^
                    ((long long)(krylov_ff ? 1 : 0) << 38) ^
                    ((long long)o.cheb_steps << 30) ^ ((long long)o.vcycles << 24) ^
                    ((long long)o.smooth_pre << 16) ^ ((long long)o.smooth_post << 8) ^
                    ((long long)(fused ? 1 : 0) << 4) ^ ((long long)o.kernel_flags << 48) ^
                    (long long)(size_t)stream;
    bool graphs = use_graphs && !prof_on && !phases_on;
    if (!graphs) {
      arnoldi_body(o, j, stride, len, tri);
      return;
    }
    if (key != gkey) {
      drop_graphs();
      gkey = key;
    }
    if ((int)gexec.size() <= j) {
      gexec.resize(j + 1, nullptr);
      gruns.resize(j + 1, 0);
    }
    if (!gexec[j] && gruns[j] >= 1) {
      cudaGraph_t graph = nullptr;
      long long before = launches_thread();
      CK(cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal));
      try {
        arnoldi_body(o, j, stride, len, tri);
      } catch (...) {
        // leave the stream usable: end (and drop) the partial capture, then report
        cudaGraph_t partial = nullptr;
        cudaStreamEndCapture(stream, &partial);
        if (partial) cudaGraphDestroy(partial);
        cudaGetLastError();
        count_launches(before - launches_thread());
        throw;
      }
      CK(cudaStreamEndCapture(stream, &graph));
      // captured launches do not run now: count them at each replay instead
      gcount.resize(j + 1, 0);
      gcount[j] = launches_thread() - before;
      count_launches(-gcount[j]);
      cudaGraphExec_t ex = nullptr;
      cudaError_t e = cudaGraphInstantiate(&ex, graph, 0);
      cudaGraphDestroy(graph);
      CK(e);
      gexec[j] = ex;
    }
    ++gruns[j];
    if (gexec[j]) {
      count_launches(gcount[j]);
      CK(cudaGraphLaunch(gexec[j], stream));
    } else {
      arnoldi_body(o, j, stride, len, tri);
    }
  }

  std::vector<long long> gcount;  // kernels inside each captured Arnoldi step

  // ------------------------------------------------------------------------
  // Right-preconditioned flexible GMRES with classical Gram-Schmidt applied
  // twice; restarts every o.restart iterations. x0 = 0. The residual estimate
  // |g_{j+1}| is the unpreconditioned residual norm ||b - A x_j||.
  // ------------------------------------------------------------------------
  void fgmres(const ipm_options& o, const double* b, double* x, int tri, int* iters,
              double* relres) {
    long long len = 4 * F();
    long long stride = len;
    int m = o.restart;
    double nb = norm(b, len);
    CK(cudaMemsetAsync(x, 0, sizeof(double) * len, stream));
    *iters = 0;
    *relres = 0.0;
    if (nb == 0.0) return;
    double tol = o.krylov_tol * nb;
    std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), gv(m + 1), y(m);
    // mixed precision: float-float Arnoldi basis (kernel_flags bit 5 keeps it in FP64)
    krylov_ff = o.precision == IPM_PREC_MIXED && !(o.kernel_flags & 32);
    // the operator writes interior nodes only: when the basis changes layout, the other
    // entries of the old one would read as nonzero in the new one
    const int lay = krylov_ff ? 1 : 0;
    if (vlayout != -1 && vlayout != lay)
      CK(cudaMemsetAsync(V, 0, sizeof(double) * (size_t)(vcap + 1) * len, stream));
    vlayout = lay;
    int total = 0;
    bool first = true;
    double res = nb;
    while (true) {
      const double* r0 = b;
      if (!first) {
        newton_apply(x, ktmp);
        launch_axpby(ktmp, b, 1.0, -1.0, len, stream);  // ktmp = b - A x
        r0 = ktmp;
        res = norm(ktmp, len);
        if (res <= tol || total >= o.max_krylov) break;
      }
      if (krylov_ff) launch_to_ff((float*)V, r0, 1.0 / res, len, stream);
      else launch_axpby(V, r0, 1.0 / res, 0.0, len, stream);
      std::fill(gv.begin(), gv.end(), 0.0);
      gv[0] = res;
      int j = 0;
      bool done = false;
      for (; j < m && total < o.max_krylov; ++j) {
        arnoldi_step(o, j, stride, len, tri);
        sync();
        ++total;
        double* h = &H[(size_t)j * (m + 1)];
        for (int i = 0; i <= j; ++i) h[i] = hbuf[i] + hbuf[(kMaxRestart + 2) + i];
        double hn = std::sqrt(hbuf[2 * (kMaxRestart + 2)]);
        h[j + 1] = hn;
        if (!std::isfinite(hn)) throw IpmError{IPM_EBREAKDOWN, "non-finite Krylov vector"};
        for (int i = 0; i < j; ++i) {
          double t = cs[i] * h[i] + sn[i] * h[i + 1];
          h[i + 1] = -sn[i] * h[i] + cs[i] * h[i + 1];
          h[i] = t;
        }
        double rr = std::hypot(h[j], h[j + 1]);
        if (rr == 0.0) throw IpmError{IPM_EBREAKDOWN, "GMRES breakdown (singular Hessenberg)"};
        cs[j] = h[j] / rr;
        sn[j] = h[j + 1] / rr;
        h[j] = rr;
        h[j + 1] = 0.0;
        gv[j + 1] = -sn[j] * gv[j];
        gv[j] = cs[j] * gv[j];
        res = std::fabs(gv[j + 1]);
        if (res <= tol || hn == 0.0) {
          ++j;
          done = true;
          break;
        }
      }
      // y = R^{-1} g, x += Z y
      for (int i = j - 1; i >= 0; --i) {
        double t = gv[i];
        for (int k = i + 1; k < j; ++k) t -= H[(size_t)k * (m + 1) + i] * y[k];
        y[i] = t / H[(size_t)i * (m + 1) + i];
      }
      CK(cudaMemcpyAsync(kdev + 3 * (kMaxRestart + 2), y.data(), sizeof(double) * j,
                         cudaMemcpyHostToDevice, stream));
      launch_axpy_multi(x, Z, stride, j, kdev + 3 * (kMaxRestart + 2), 1.0, len, stream);
      sync();  // y lives on the host stack
      first = false;
      if (done || total >= o.max_krylov) break;
    }
    newton_apply(x, ktmp);
    launch_axpby(ktmp, b, 1.0, -1.0, len, stream);
    *relres = norm(ktmp, len) / nb;
    *iters = total;
  }

  // ------------------------------------------------------------------------
  // Preconditioned MINRES (Paige-Saunders) with P = P_D SPD; the unpreconditioned
  // residual r = b - A x is carried along through A w recurrences.
  // ------------------------------------------------------------------------
  double dot(const double* a, const double* b, long long len) {
    launch_dot(a, b, len, part, dout, stream);
    fetch(dout, 1);
    return hbuf[0];
  }

  // MINRES with P_D. The all-FP64 path runs it once to krylov_tol. On the mixed path the
  // preconditioner (FP32 Chebyshev, z-block and V-cycles) is symmetric only to FP32 accuracy,
  // which bounds the residual MINRES's recurrences can certify; FP64 iterative refinement
  // restores the tolerance: the true residual r = b - A x in FP64, a MINRES solve of
  // A d = r to a moderate relative tolerance, x += d, until ||r|| <= krylov_tol ||b||.
  void minres(const ipm_options& o, const double* b, double* x, int* iters, double* relres) {
    const long long len = 4 * F();
    const bool refine = o.precision == IPM_PREC_MIXED && !(o.kernel_flags & 256);
    double nb = norm(b, len);
    *iters = 0;
    *relres = 0.0;
    if (nb == 0.0) {
      CK(cudaMemsetAsync(x, 0, sizeof(double) * len, stream));
      return;
    }
    if (!refine) {
      *iters = minres_core(o, b, x, o.krylov_tol * nb, o.max_krylov);
    } else {
      double* rr = mr[13];
      double* d = mr[14];
      CK(cudaMemsetAsync(x, 0, sizeof(double) * len, stream));
      launch_axpby(rr, b, 1.0, 0.0, len, stream);
      double res = nb;
      int total = 0;
      const double tol = o.krylov_tol * nb;
      for (int sweep = 0; sweep < kMaxRefine && total < o.max_krylov && res > tol; ++sweep) {
        // inner tolerance: kRefineInner relative to the current residual, not below the target
        const double inner = std::max(tol, kRefineInner * res);
        total += minres_core(o, rr, d, inner, o.max_krylov - total);
        launch_axpby(x, d, 1.0, 1.0, len, stream);
        newton_apply(x, rr);
        launch_axpby(rr, b, 1.0, -1.0, len, stream);  // rr = b - A x
        const double nr = norm(rr, len);
        if (!std::isfinite(nr)) throw IpmError{IPM_EBREAKDOWN, "non-finite refinement residual"};
        if (nr >= res) {  // no progress: keep the previous iterate and stop
          launch_axpby(x, d, -1.0, 1.0, len, stream);
          break;
        }
        res = nr;
      }
      *iters = total;
    }
    newton_apply(x, ktmp);
    launch_axpby(ktmp, b, 1.0, -1.0, len, stream);
    *relres = norm(ktmp, len) / nb;
  }

  static constexpr int kMaxRefine = 12;
  static constexpr double kRefineInner = 1e-4;

  // preconditioned MINRES for A x = b from x = 0 until the recurrence residual is below
  // tol_abs or after max_it iterations; returns the iterations taken
  int minres_core(const ipm_options& o, const double* b, double* x, double tol_abs, int max_it) {
    long long len = 4 * F();
    double *v_prev = mr[0], *v_cur = mr[1], *v_next = mr[2], *z_cur = mr[3], *z_next = mr[4];
    double *w_prev = mr[5], *w_cur = mr[6], *w_next = mr[7], *Az = mr[8];
    double *aw_prev = mr[9], *aw_cur = mr[10], *aw_next = mr[11], *r = mr[12];
    CK(cudaMemsetAsync(x, 0, sizeof(double) * len, stream));
    for (double* p : {v_prev, w_prev, w_cur, aw_prev, aw_cur})
      CK(cudaMemsetAsync(p, 0, sizeof(double) * len, stream));
    launch_axpby(r, b, 1.0, 0.0, len, stream);
    launch_axpby(v_cur, b, 1.0, 0.0, len, stream);
    double nb = norm(b, len);
    if (nb == 0.0) return 0;
    precond(v_cur, z_cur, 0, o);
    double gam = std::sqrt(dot(z_cur, v_cur, len));
    double gam_prev = 1.0, eta = gam;
    double s_prev = 0, s_cur = 0, c_prev = 1, c_cur = 1;
    double tol = tol_abs;
    double res = nb;
    int j = 0;
    while (j < max_it) {
      ++j;
      launch_axpby(z_cur, z_cur, 1.0 / gam, 0.0, len, stream);
      newton_apply(z_cur, Az);
      double delta = dot(Az, z_cur, len);
      launch_lincomb3(v_next, 1.0, Az, -delta / gam, v_cur, -gam / gam_prev, v_prev, len, stream);
      precond(v_next, z_next, 0, o);
      double g2 = dot(z_next, v_next, len);
      if (!(g2 >= 0.0)) throw IpmError{IPM_EBREAKDOWN, "preconditioner not positive definite"};
      double gam_next = std::sqrt(g2);
      double a0 = c_cur * delta - c_prev * s_cur * gam;
      double a1 = std::sqrt(a0 * a0 + gam_next * gam_next);
      double a2 = s_cur * delta + c_prev * c_cur * gam;
      double a3 = s_prev * gam;
      if (a1 == 0.0) throw IpmError{IPM_EBREAKDOWN, "MINRES breakdown"};
      double c_next = a0 / a1, s_next = gam_next / a1;
      launch_lincomb3(w_next, 1.0 / a1, z_cur, -a3 / a1, w_prev, -a2 / a1, w_cur, len, stream);
      launch_lincomb3(aw_next, 1.0 / a1, Az, -a3 / a1, aw_prev, -a2 / a1, aw_cur, len, stream);
      launch_axpby(x, w_next, c_next * eta, 1.0, len, stream);
      launch_axpby(r, aw_next, -c_next * eta, 1.0, len, stream);
      eta = -s_next * eta;
      res = norm(r, len);
      std::swap(v_prev, v_cur);
      std::swap(v_cur, v_next);
      std::swap(z_cur, z_next);
      gam_prev = gam;
      gam = gam_next;
      std::swap(w_prev, w_cur);
      std::swap(w_cur, w_next);
      std::swap(aw_prev, aw_cur);
      std::swap(aw_cur, aw_next);
      c_prev = c_cur;
      c_cur = c_next;
      s_prev = s_cur;
      s_cur = s_next;
      if (!std::isfinite(res)) throw IpmError{IPM_EBREAKDOWN, "non-finite MINRES residual"};
      if (res <= tol || gam == 0.0) break;
    }
    return j;
  }

  void krylov(const ipm_options& o, const double* b, double* x, int* iters, double* relres) {
    if (o.krylov == IPM_KRYLOV_GMRES_PT) fgmres(o, b, x, 1, iters, relres);
    else minres(o, b, x, iters, relres);
  }

  // ------------------------------------------------------------------------
  // Algorithm A.1
  // ------------------------------------------------------------------------
  void residual_row(double mu, int k, double aP, double aD, int kit, double krr) {
    launch_residuals(g, problem(), bounds(), st, mu, part, dout, stream);
    fetch(dout, 8);
    double* q = hbuf;
    double xp = std::sqrt(q[0]), xd = std::sqrt(q[1]), xc = std::sqrt(q[2]);
    double Q = 0.5 * (q[4] - 2.0 * q[5] + c0) + 0.5 * alpha * q[6] + beta * lumped_mass(g) * q[7];
    double rp = xp / (1.0 + nf + ncy);
    double rd = xd / (1.0 + ncy + beta * nd);
    mean_prod = nbounds > 0 ? q[3] / nbounds : 0.0;
    double rc = mean_prod / (1.0 + std::fabs(Q));
    double kkt = std::max(rp, std::max(rd, rc));
    double row[kHistCols] = {(double)k, mu, xp, xd, xc, kkt, aP, aD, (double)kit, krr};
    hist.insert(hist.end(), row, row + kHistCols);
  }

  // After a breakdown, a non-finite scalar (a norm, a step length) may have been applied to
  // whole arrays, so boundary and padding entries, which kernels read as zero but never
  // write, can hold NaN. Zero every work array; the problem data (bounds, data vectors,
  // Dirichlet lift, operator coefficients) are kept.
  void scrub_work() {
    std::vector<const void*> keep = {ya, yb, zbw, zbv, cy, fvec, glift, ydbuf, fbuf};
    for (const OpL& op : lvop) {
      keep.push_back(op.coef);
      keep.push_back(op.coef32);
    }
    for (size_t i = 0; i < allocs.size(); ++i) {
      if (std::find(keep.begin(), keep.end(), allocs[i]) != keep.end()) continue;
      CK(cudaMemsetAsync(allocs[i], 0, alloc_bytes[i], stream));
    }
    sync();
  }

  void apply_flags(const ipm_options& o) {
    fused = (o.kernel_flags & 1) == 0;
    ff_outer = (o.kernel_flags & 16) == 0;
    nu_fits = o.smooth_pre <= 8 && o.smooth_post <= 8;
    use_graphs = (o.kernel_flags & 2) == 0;
    use_mid_cycle = (o.kernel_flags & 128) != 0;
    autotune = (o.kernel_flags & 512) == 0;
    ff_operator = (o.kernel_flags & 1024) == 0;
  }

  int solve(const ipm_options& o, ipm_report* rep) {
    apply_flags(o);
    if (!has_data) throw IpmError{IPM_ESTATE, "ipm_set_data must precede ipm_solve"};
    if (o.restart < 1 || o.restart > kMaxRestart) throw IpmError{IPM_EINVAL, "restart out of range [1, 100]"};
    if (o.cheb_steps < 1 || o.vcycles < 1 || o.smooth_pre < 0 || o.smooth_post < 0 ||
        !(o.sigma > 0 && o.sigma < 1) || !(o.alpha0 > 0 && o.alpha0 < 1) || !(o.mu0 > 0) ||
        o.max_krylov < 1 || o.max_ipm < 0 || o.mu_rule < 0 || o.mu_rule > 1)
      throw IpmError{IPM_EINVAL, "invalid solver options"};
    if (heat() && o.krylov != IPM_KRYLOV_GMRES_PT)
      throw IpmError{IPM_EINVAL, "the heat equation is solved with GMRES + P_T"};
    if (g.obs && (o.krylov != IPM_KRYLOV_GMRES_PT || o.precision != IPM_PREC_FP64))
      throw IpmError{IPM_EINVAL, "partial observation is solved with GMRES + P_Pi in FP64"};
    if (o.smooth_pre != o.smooth_post && o.krylov == IPM_KRYLOV_MINRES_PD)
      throw IpmError{IPM_EINVAL, "MINRES needs a symmetric V-cycle (smooth_pre == smooth_post)"};
    auto t0 = std::chrono::steady_clock::now();
    ensure_krylov(o);
    last_precision = o.precision;
    hist.clear();
    double mu = o.mu0;
    launch_init_state(g, bounds(), st, mu, stream);
    residual_row(mu, 0, 0.0, 0.0, 0, 0.0);
    int k = 0, status = IPM_OK, ktot = 0;
    double krr_max = 0.0;
    while (true) {
      const double* h = &hist[hist.size() - kHistCols];
      bool stop;
      if (o.stop == IPM_STOP_FIXED) stop = k >= o.fixed_iters;
      else if (o.stop == IPM_STOP_PAPER) stop = h[2] <= o.eps_p && h[3] <= o.eps_d && h[4] <= o.eps_c;
      else stop = h[5] <= o.kkt_tol;
      if (stop) break;
      if (k >= o.max_ipm) {
        status = IPM_ENOTCONV;
        break;
      }
      double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
      if (o.time_limit_s > 0 && el > o.time_limit_s) {
        status = IPM_ETIMEOUT;
        break;
      }
      mu = o.mu_rule == 1 ? o.sigma * mean_prod : o.sigma * mu;
      launch_prep(g, problem(), bounds(), st, dg, mu, rhs, o.precision == IPM_PREC_MIXED || heat(),
                  stream);
      setup_precond(o);
      int kit = 0;
      double krr = 0.0;
      krylov(o, rhs, dx, &kit, &krr);
      ktot += kit;
      krr_max = std::max(krr_max, krr);
      launch_steplen(g, bounds(), st, dx, mu, o.alpha0, o.common_step, part, sc, stream);
      launch_update(g, bounds(), st, dx, mu, sc, stream);
      ++k;
      fetch(sc, 2);
      double aP = hbuf[0], aD = hbuf[1];
      residual_row(mu, k, aP, aD, kit, krr);
      if (!std::isfinite(hist[hist.size() - kHistCols + 5]))
        throw IpmError{IPM_EBREAKDOWN, "non-finite residuals"};
    }
    solved = true;
    if (rep) {
      const double* h = &hist[hist.size() - kHistCols];
      rep->status = status;
      rep->ipm_iters = k;
      rep->krylov_iters_total = ktot;
      rep->kkt_rel = h[5];
      rep->xi_p = h[2];
      rep->xi_d = h[3];
      rep->xi_c = h[4];
      rep->mu = mu;
      rep->krylov_relres_max = krr_max;
      rep->seconds =
          std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
    return status;
  }

  void get(int which, double* out, size_t len, bool device) const {
    if (!solved) throw IpmError{IPM_ESTATE, "no solution yet"};
    if ((long long)len != nn()) throw IpmError{IPM_EINVAL, "output length must be n^d"};
    ipm_solver* self = const_cast<ipm_solver*>(this);
    const double* src = which == 0 ? st.y : which == 2 ? st.p : nullptr;
    double* tgt = device ? out : self->dense;
    if (which == 1) {
      // u = w - v into the dense scratch through ktmp
      launch_lincomb3(self->ktmp, 1.0, st.w, -1.0, st.v, 0.0, nullptr, F(), stream);
      src = self->ktmp;
    }
    launch_unpack(g, src, which == 0 ? glift : nullptr, tgt, stream);
    if (!device)
      CK(cudaMemcpyAsync(out, self->dense, sizeof(double) * nn(), cudaMemcpyDeviceToHost, stream));
    self->sync();
  }
};

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
namespace {
template <typename Fn>
int guarded(ipm_solver* s, Fn fn) {
  try {
    return fn();
  } catch (const IpmError& e) {
    if (s) s->err = e.msg;
    return e.code;
  } catch (const std::exception& e) {
    if (s) s->err = e.what();
    return IPM_ECUDA;
  }
}
thread_local std::string g_create_err;
}  // namespace

extern "C" {

void ipm_default_options(ipm_options* o) {
  if (!o) return;
  o->precision = IPM_PREC_FP64;
  o->krylov = IPM_KRYLOV_GMRES_PT;
  o->stop = IPM_STOP_PAPER;
  o->sigma = 0.2;
  o->alpha0 = 0.995;
  o->eps_p = o->eps_d = o->eps_c = 1e-6;
  o->mu0 = 1.0;
  o->kkt_tol = 1e-6;
  o->krylov_tol = 1e-10;
  o->cheb_steps = 20;
  o->vcycles = 3;
  o->smooth_pre = 5;
  o->smooth_post = 5;
  o->max_ipm = 100;
  o->max_krylov = 200;
  o->restart = 50;
  o->fixed_iters = 0;
  o->time_limit_s = 0.0;
  o->common_step = 0;
  o->mu_rule = 0;
  o->kernel_flags = 0;
}

int ipm_create(const ipm_grid* grid, const ipm_pde* pde, double alpha, double beta,
               const ipm_bounds* bounds, ipm_solver** out) {
  if (!out) return IPM_EINVAL;
  *out = nullptr;
  ipm_solver* s = new ipm_solver();
  int rc = guarded(s, [&] {
    s->create(grid, pde, alpha, beta, bounds);
    return IPM_OK;
  });
  if (rc != IPM_OK) {
    g_create_err = s->err;
    s->release();
    delete s;
    return rc;
  }
  *out = s;
  return IPM_OK;
}

int ipm_reset(ipm_solver* s, double alpha, double beta, const ipm_bounds* bounds) {
  if (!s) return IPM_EINVAL;
  return guarded(s, [&] {
    s->reset(alpha, beta, bounds);
    return IPM_OK;
  });
}

size_t ipm_device_bytes(const ipm_solver* s) { return s ? s->bytes : 0; }

int ipm_set_stream(ipm_solver* s, void* stream) {
  if (!s) return IPM_EINVAL;
  cudaStream_t next = stream ? (cudaStream_t)stream : s->own;
  // work already enqueued on the previous stream (zeroing of new buffers, an unfinished
  // device-pointer call) completes before anything enqueued on the next one
  if (next != s->stream && cudaStreamSynchronize(s->stream) != cudaSuccess) {
    cudaGetLastError();
    return IPM_ECUDA;
  }
  s->stream = next;
  return IPM_OK;
}

int ipm_set_data(ipm_solver* s, const double* yd, const double* f, const double* g) {
  if (!s) return IPM_EINVAL;
  return guarded(s, [&] {
    s->set_data(yd, f, g, false);
    return IPM_OK;
  });
}

int ipm_set_data_device(ipm_solver* s, const double* yd, const double* f, const double* g) {
  if (!s) return IPM_EINVAL;
  return guarded(s, [&] {
    s->set_data(yd, f, g, true);
    return IPM_OK;
  });
}

int ipm_solve(ipm_solver* s, const ipm_options* opt, ipm_report* rep) {
  if (!s) return IPM_EINVAL;
  ipm_options o;
  if (opt) o = *opt;
  else ipm_default_options(&o);
  int rc = guarded(s, [&] { return s->solve(o, rep); });
  if (rc == IPM_EBREAKDOWN) {
    // leave the solver usable for new data: clear what the non-finite values touched
    int rs = guarded(s, [&] {
      s->scrub_work();
      return IPM_OK;
    });
    if (rs != IPM_OK) return rs;
  }
  return rc;
}

static int get_common(const ipm_solver* s, int which, double* out, size_t len, bool dev) {
  if (!s || !out) return IPM_EINVAL;
  ipm_solver* m = const_cast<ipm_solver*>(s);
  return guarded(m, [&] {
    s->get(which, out, len, dev);
    return IPM_OK;
  });
}
int ipm_get_state(const ipm_solver* s, double* y, size_t len) { return get_common(s, 0, y, len, false); }
int ipm_get_control(const ipm_solver* s, double* u, size_t len) { return get_common(s, 1, u, len, false); }
int ipm_get_adjoint(const ipm_solver* s, double* p, size_t len) { return get_common(s, 2, p, len, false); }
int ipm_get_state_device(const ipm_solver* s, double* y, size_t len) { return get_common(s, 0, y, len, true); }
int ipm_get_control_device(const ipm_solver* s, double* u, size_t len) { return get_common(s, 1, u, len, true); }
int ipm_get_adjoint_device(const ipm_solver* s, double* p, size_t len) { return get_common(s, 2, p, len, true); }

int ipm_get_history(const ipm_solver* s, double* rows, int max_rows, int* n_rows) {
  if (!s || !n_rows) return IPM_EINVAL;
  int nr = (int)(s->hist.size() / kHistCols);
  *n_rows = nr;
  if (rows && max_rows > 0)
    std::memcpy(rows, s->hist.data(), sizeof(double) * kHistCols * std::min(nr, max_rows));
  return IPM_OK;
}

void ipm_destroy(ipm_solver* s) {
  if (!s) return;
  if (s->stream) cudaStreamSynchronize(s->stream);
  s->release();
  delete s;
}

const char* ipm_strerror(int code) {
  switch (code) {
    case IPM_OK: return "ok";
    case IPM_EINVAL: return "invalid argument";
    case IPM_ENOMEM: return "out of device memory";
    case IPM_ENOTCONV: return "iteration limit reached before convergence";
    case IPM_EBREAKDOWN: return "Krylov breakdown or non-finite values";
    case IPM_ETIMEOUT: return "time limit reached";
    case IPM_ECUDA: return "CUDA error";
    case IPM_ESTATE: return "call out of order";
    default: return "unknown error";
  }
}

long long ipm_launch_count(void) { return launches_total(); }

int ipm_profile_smoother(ipm_solver* s, int enable, int every) {
  if (!s || every < 1) return IPM_EINVAL;
  return guarded(s, [&] {
    s->prof_flush();
    s->prof_on = enable != 0;
    s->prof_kind = 0;
    s->prof_every = every;
    s->prof_seen = 0;
    s->prof_ms = 0.0;
    s->prof_count = 0;
    s->prof_zero = 0;
    return IPM_OK;
  });
}

int ipm_profile_phases(ipm_solver* s, int enable, double* ms, long long* counts, int nphases) {
  if (!s) return IPM_EINVAL;
  return guarded(s, [&] {
    s->prof_flush();
    for (int i = 0; i < nphases && i < 16; ++i) {
      if (ms) ms[i] = s->ph_ms[i];
      if (counts) counts[i] = s->ph_count[i];
    }
    if (enable >= 0) {
      s->phases_on = enable != 0;
      for (int i = 0; i < 16; ++i) {
        s->ph_ms[i] = 0.0;
        s->ph_count[i] = 0;
      }
    }
    return IPM_OK;
  });
}

int ipm_profile_read(ipm_solver* s, double* total_ms, long long* launches, double* bytes_per_launch) {
  if (!s) return IPM_EINVAL;
  return guarded(s, [&] {
    s->prof_flush();
    if (total_ms) *total_ms = s->prof_ms;
    if (launches) *launches = s->prof_count;
    // algorithmic bytes of one sampled finest-level launch, per unknown: fused 2D kernel
    // (nu sweeps + residual + restriction) reads x, b, m and writes x and a quarter-size
    // coarse right-hand side (4.25 values; 3.25 when it starts from zero and reads no x);
    // a single sweep reads x, b, m, jinv and writes x (5)
    long long m = s->g.n - 2;
    long long unknowns = s->g.dim == 3 ? m * m * m : m * m;
    double zfrac = s->prof_count ? (double)s->prof_zero / (double)s->prof_count : 0.0;
    double vals = s->fused_mg() ? 4.25 - zfrac : 5.0;
    double word = s->last_precision == IPM_PREC_MIXED ? 4.0 : 8.0;
    if (bytes_per_launch) *bytes_per_launch = vals * (double)unknowns * word;
    return IPM_OK;
  });
}

int ipm_profile_kernel(ipm_solver* s, int kind, int enable, int every) {
  if (!s || kind < 0 || kind > 4 || every < 1) return IPM_EINVAL;
  return guarded(s, [&] {
    s->prof_flush();
    s->prof_on = enable != 0;
    s->prof_kind = kind;
    s->prof_every = every;
    s->prof_seen = 0;
    s->prof_ms = 0.0;
    s->prof_count = 0;
    s->prof_zero = 0;
    s->prof_bp_sum = 0.0;
    s->prof_bo_sum = 0.0;
    return IPM_OK;
  });
}

int ipm_profile_kernel_read(ipm_solver* s, double* total_ms, long long* sampled, long long* calls,
                            double* bytes_pass, double* bytes_once) {
  if (!s) return IPM_EINVAL;
  return guarded(s, [&] {
    s->prof_flush();
    const double k = s->prof_count > 0 ? (double)s->prof_count : 1.0;
    if (total_ms) *total_ms = s->prof_ms;
    if (sampled) *sampled = s->prof_count;
    if (calls) *calls = s->prof_seen;
    if (bytes_pass) *bytes_pass = s->prof_bp_sum / k;
    if (bytes_once) *bytes_once = s->prof_bo_sum / k;
    return IPM_OK;
  });
}

int ipm_set_observation(ipm_solver* s, const double* lo, const double* hi) {
  if (!s || (!lo) != (!hi)) return IPM_EINVAL;
  return guarded(s, [&] {
    s->set_observation(lo, hi);
    return IPM_OK;
  });
}

int ipm_tuning_report(char* buf, size_t len) { return mg2_tune_report(buf, len); }

int ipm_tuning_set(int kernel, int n, int shape) {
  return mg2_tune_set(kernel, n, shape) == 0 ? IPM_OK : IPM_EINVAL;
}

const char* ipm_last_error(const ipm_solver* s) {
  return s ? s->err.c_str() : g_create_err.c_str();
}

// ---------------------------------------------------------------------------
// Component entry points
// ---------------------------------------------------------------------------
int ipm_newton_apply_device(ipm_solver* s, const double* ty, const double* tw, const double* tv,
                            const double* x, double* out) {
  if (!s || !ty || !tw || !tv || !x || !out) return IPM_EINVAL;
  return guarded(s, [&] {
    long long f = s->F(), m = s->nn();
    launch_pack(s->g, ty, s->dg.thy, 1, s->stream);
    launch_pack(s->g, tw, s->dg.thw, 1, s->stream);
    launch_pack(s->g, tv, s->dg.thv, 1, s->stream);
    for (int b = 0; b < 4; ++b) launch_pack(s->g, x + b * m, s->rhs + b * f, 1, s->stream);
    s->newton_apply(s->rhs, s->dx);
    for (int b = 0; b < 4; ++b) launch_unpack(s->g, s->dx + b * f, nullptr, out + b * m, s->stream);
    s->sync();
    return IPM_OK;
  });
}

int ipm_newton_apply_ff_device(ipm_solver* s, const double* ty, const double* tw,
                               const double* tv, const double* x, double* out) {
  if (!s || !ty || !tw || !tv || !x || !out) return IPM_EINVAL;
  return guarded(s, [&] {
    if (!newton_apply_ff2_ok(s->g, s->problem()))
      throw IpmError{IPM_EINVAL, "the float-float operator covers 2D Poisson without observation"};
    long long f = s->F(), m = s->nn();
    launch_pack(s->g, ty, s->dg.thy, 1, s->stream);
    launch_pack(s->g, tw, s->dg.thw, 1, s->stream);
    launch_pack(s->g, tv, s->dg.thv, 1, s->stream);
    launch_to_ff(s->dg.thyff, s->dg.thy, 1.0, f, s->stream);  // high plane, then low plane
    for (int b = 0; b < 4; ++b) launch_pack(s->g, x + b * m, s->rhs + b * f, 1, s->stream);
    float* ff = reinterpret_cast<float*>(s->dx);  // 8 f floats: high parts, then low parts
    launch_newton_apply_ff2(s->g, s->problem(), s->dg, s->rhs, ff, s->stream);
    launch_from_ff(s->ktmp, ff, 4 * f, s->stream);
    for (int b = 0; b < 4; ++b) launch_unpack(s->g, s->ktmp + b * f, nullptr, out + b * m, s->stream);
    s->sync();
    return IPM_OK;
  });
}

static void load_diags(ipm_solver* s, const double* ty, const double* tw, const double* tv) {
  launch_pack(s->g, ty, s->dg.thy, 1, s->stream);
  launch_pack(s->g, tw, s->dg.thw, 1, s->stream);
  launch_pack(s->g, tv, s->dg.thv, 1, s->stream);
  launch_mhat(s->g, s->alpha, mass_diag(s->g), s->dg.thy, s->dg.thw, s->dg.thv, s->dg.mh,
              s->dg.thy32, s->dg.mh32, s->stream);
  launch_to_float2(s->g, s->dg.thw, s->dg.thv, s->dg.thw32, s->dg.thv32, s->stream);
  launch_to_ff(s->dg.thyff, s->dg.thy, 1.0, s->F(), s->stream);
}

int ipm_precond_apply_device(ipm_solver* s, const ipm_options* opt, int tri, const double* ty,
                             const double* tw, const double* tv, const double* r, double* z) {
  if (!s || !ty || !tw || !tv || !r || !z) return IPM_EINVAL;
  ipm_options o;
  if (opt) o = *opt;
  else ipm_default_options(&o);
  return guarded(s, [&] {
    s->apply_flags(o);
    long long f = s->F(), m = s->nn();
    load_diags(s, ty, tw, tv);
    s->setup_precond(o);
    for (int b = 0; b < 4; ++b) launch_pack(s->g, r + b * m, s->rhs + b * f, 1, s->stream);
    // the mixed FGMRES path applies P_T to float-float Krylov vectors: take that path too
    s->krylov_ff = o.precision == IPM_PREC_MIXED && !(o.kernel_flags & 32);
    if (s->precond_ff_ok(o, tri)) {
      float* v = (float*)s->ktmp;
      launch_to_ff(v, s->rhs, 1.0, 4 * f, s->stream);
      s->precond_ff(v, s->dx, o);
    } else {
      s->precond(s->rhs, s->dx, tri, o);
    }
    for (int b = 0; b < 4; ++b) launch_unpack(s->g, s->dx + b * f, nullptr, z + b * m, s->stream);
    s->sync();
    return IPM_OK;
  });
}

int ipm_chebyshev_device(ipm_solver* s, int steps, const double* ty, const double* b, double* x) {
  if (!s || !ty || !b || !x || steps < 1) return IPM_EINVAL;
  return guarded(s, [&] {
    launch_pack(s->g, ty, s->dg.thy, 1, s->stream);
    launch_pack(s->g, b, s->rhs, 1, s->stream);
    s->cheb_apply<double, double>(s->rhs, s->dg.thy, s->dx, steps, s->cheb64);
    launch_unpack(s->g, s->dx, nullptr, x, s->stream);
    s->sync();
    return IPM_OK;
  });
}

int ipm_vcycle_device(ipm_solver* s, const ipm_options* opt, int tr, const double* m,
                      const double* b, double* x) {
  if (!s || !m || !b || !x) return IPM_EINVAL;
  ipm_options o;
  if (opt) o = *opt;
  else ipm_default_options(&o);
  return guarded(s, [&] {
    s->apply_flags(o);
    launch_pack(s->g, m, s->dg.mh, 1, s->stream);
    if (o.precision == IPM_PREC_MIXED) {
      // the preconditioner's mixed solve: FP32 cycles, outer residual and iterate in
      // float-float (2D Poisson) or FP64
      launch_convert<double, float>(s->g, s->dg.mh, s->dg.mh32, s->stream);
      s->mg_setup_mixed();
      launch_pack(s->g, b, s->mgb64, 1, s->stream);
      double* xr = s->mg64.lv[0].x[0];
      s->mg_solve_mixed(s->mgb64, xr, tr, o);
      launch_unpack(s->g, xr, nullptr, x, s->stream);
    } else {
      s->mg_setup(s->mg64, s->dg.mh);
      launch_pack(s->g, b, s->mg64.lv[0].b, 1, s->stream);
      double* xr = s->mg_solve(s->mg64, tr, o);
      launch_unpack(s->g, xr, nullptr, x, s->stream);
    }
    s->sync();
    return IPM_OK;
  });
}

int ipm_newton_step_device(ipm_solver* s, const ipm_options* opt, const double* const* it,
                           double mu, double* dxo, int* iters, double* relres) {
  if (!s || !it || !dxo) return IPM_EINVAL;
  ipm_options o;
  if (opt) o = *opt;
  else ipm_default_options(&o);
  return guarded(s, [&] {
    s->apply_flags(o);
    if (!s->has_data) throw IpmError{IPM_ESTATE, "ipm_set_data must come first"};
    double* dst[10] = {s->st.y, s->st.w, s->st.v, s->st.p, s->st.lya,
                       s->st.lyb, s->st.lwa, s->st.lwb, s->st.lva, s->st.lvb};
    for (int q = 0; q < 10; ++q) launch_pack(s->g, it[q], dst[q], 1, s->stream);
    s->ensure_krylov(o);
    launch_prep(s->g, s->problem(), s->bounds(), s->st, s->dg, mu, s->rhs,
                o.precision == IPM_PREC_MIXED, s->stream);
    s->setup_precond(o);
    int kit = 0;
    double krr = 0;
    s->krylov(o, s->rhs, s->dx, &kit, &krr);
    long long f = s->F(), m = s->nn();
    for (int b = 0; b < 4; ++b) launch_unpack(s->g, s->dx + b * f, nullptr, dxo + b * m, s->stream);
    s->sync();
    if (iters) *iters = kit;
    if (relres) *relres = krr;
    return IPM_OK;
  });
}

}  // extern "C"
