// Shared device-side definitions: grid layout, Q1 stencils, reductions.
//
// Layout: every nodal field lives on the full uniform grid of the unit square
// (cube), boundary nodes included, x fastest, rows padded to `pitch` elements
// (a multiple of 32) so that rows start on 128-byte (FP32) / 256-byte (FP64)
// boundaries. Boundary and padding entries of vectors the Krylov solvers see
// are kept at zero, so whole-field reductions equal sums over the unknowns.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include <cstddef>

#define IPM_HD __host__ __device__ __forceinline__
#define IPM_D __device__ __forceinline__

// Every member has a default so that a descriptor filled in field by field never carries
// stack contents into a kernel (the heat and observation members select stencil branches).
struct GridDesc {
  int dim = 2;          // 2 or 3
  int n = 0;            // nodes per direction, boundary included
  int pitch = 0;        // elements per row
  long long plane = 0;  // elements per z-plane (pitch * n)
  long long field = 0;  // elements per field (plane for 2D, plane * n for 3D)
  double h = 0.0;       // mesh size 1/(n-1)
  // Space-time layout of the all-at-once heat equation (Section 3.4): a 2D grid of n^2
  // nodes per time level stored as the z-planes of a dim-3 grid, plane k = time t_k
  // (plane 0 the initial state, planes 1 .. n-2 the unknown levels, plane n-1 unused),
  // with the time-level masses tau M and the backward-Euler operator below.
  int heat = 0;         // 0, or 1 for the space-time layout
  double tau = 0.0;     // time step (heat layout)
  // Partial observation (the subsection on partial observations): per element, indexed by
  // the element's lowest-corner node, 1 where the tracking term integrates, else 0; null =
  // the whole domain. Only the tracking mass M_s of the state row uses it.
  const float* obs = nullptr;
};

IPM_HD long long node_index(const GridDesc& g, int i, int j, int k) {
  return (long long)k * g.plane + (long long)j * g.pitch + i;
}

inline GridDesc make_grid(int dim, int n) {
  GridDesc g;
  g.dim = dim;
  g.n = n;
  g.pitch = (n + 31) / 32 * 32;
  g.plane = (long long)g.pitch * n;
  g.field = dim == 2 ? g.plane : g.plane * n;
  g.h = 1.0 / (n - 1);
  g.heat = 0;
  g.tau = 0.0;
  g.obs = nullptr;
  return g;
}

// The space-time grid of the heat equation: n^2 nodes per level, n - 2 time levels of
// size tau.
inline GridDesc make_heat_grid(int n, double tau) {
  GridDesc g = make_grid(3, n);
  g.heat = 1;
  g.tau = tau;
  return g;
}

// Launch shape for one thread per interior node: x along rows, y across rows,
// z over interior planes (3D).
inline dim3 interior_block() { return dim3(32, 8, 1); }
inline dim3 interior_grid(const GridDesc& g) {
  int m = g.n - 2;
  return dim3((m + 31) / 32, (m + 7) / 8, g.dim == 3 ? m : 1);
}

// Maps the calling thread to an interior node; returns false for threads past the edge.
IPM_D bool interior_node(const GridDesc& g, int& i, int& j, int& k, long long& c) {
  i = 1 + blockIdx.x * blockDim.x + threadIdx.x;
  j = 1 + blockIdx.y * blockDim.y + threadIdx.y;
  k = g.dim == 3 ? 1 + (int)blockIdx.z : 0;
  if (i > g.n - 2 || j > g.n - 2) return false;
  c = node_index(g, i, j, k);
  return true;
}

// ---------------------------------------------------------------------------
// Q1 stencils on the uniform grid (interior rows of the Galerkin matrices).
// Mass:      M = M1 (x) M1 [(x) M1],  M1 = (h/6)[1 4 1]
// Stiffness: 2D  (1/3)[8 at centre, -1 at the 8 neighbours]  (independent of h)
//            3D  h [8/3 centre, 0 faces, -1/6 edges, -1/12 corners]
// Diagonals: D_M = (2h/3)^d;  stiffness diagonal 8/3 (2D), 8h/3 (3D).
// ---------------------------------------------------------------------------
// Generic forms take a load functor f(index) -> T, so that e.g. M(w - v)
// forms the difference before the stencil sum.
template <typename T, typename F>
IPM_D T row141(const F& f, long long c) {
  return f(c - 1) + T(4) * f(c) + f(c + 1);
}
template <typename T, typename F>
IPM_D T row111(const F& f, long long c) {
  return f(c - 1) + f(c) + f(c + 1);
}
// Mass action without the h^d/6^d factor.
template <typename T, typename F>
IPM_D T mass2_raw(const F& f, long long c, int p) {
  return row141<T>(f, c - p) + T(4) * row141<T>(f, c) + row141<T>(f, c + p);
}
template <typename T, typename F>
IPM_D T mass3_raw(const F& f, long long c, int p, long long pl) {
  return mass2_raw<T>(f, c - pl, p) + T(4) * mass2_raw<T>(f, c, p) + mass2_raw<T>(f, c + pl, p);
}
// 2D stiffness: (8 x_c - sum of 8 neighbours)/3 = 3 x_c - (3x3 box sum)/3.
template <typename T, typename F>
IPM_D T stiff2(const F& f, long long c, int p) {
  T box = row111<T>(f, c - p) + row111<T>(f, c) + row111<T>(f, c + p);
  return T(3) * f(c) - box * T(1.0 / 3.0);
}
// 3D stiffness without the factor h: 8/3 x_c - (1/6) edges - (1/12) corners.
template <typename T, typename F>
IPM_D T stiff3_raw(const F& f, long long c, int p, long long pl) {
  T e = f(c - p - 1) + f(c - p + 1) + f(c + p - 1) + f(c + p + 1);
  T cor = T(0);
#pragma unroll
  for (int s = -1; s <= 1; s += 2) {
    long long cc = c + s * pl;
    e += f(cc - 1) + f(cc + 1) + f(cc - p) + f(cc + p);
    cor += f(cc - p - 1) + f(cc - p + 1) + f(cc + p - 1) + f(cc + p + 1);
  }
  return T(8.0 / 3.0) * f(c) - e * T(1.0 / 6.0) - cor * T(1.0 / 12.0);
}

template <typename T>
struct Ld {  // plain load functor
  const T* __restrict__ x;
  IPM_D T operator()(long long i) const { return x[i]; }
};
template <typename T>
struct LdDiff {  // a - b
  const T* __restrict__ a;
  const T* __restrict__ b;
  IPM_D T operator()(long long i) const { return a[i] - b[i]; }
};
template <typename T, typename S>
struct LdCvt {  // load S, convert to T
  const S* __restrict__ x;
  IPM_D T operator()(long long i) const { return (T)x[i]; }
};

template <typename T>
struct Stencil {
  int dim;
  int p;
  long long pl;
  T mscale;  // h^d / 6^d (heat layout: tau h^2 / 36, the time-level mass)
  T kscale;  // 1 (2D) or h (3D)
  int heat;  // space-time layout: masses act within a time level
  T tau;
  T m2scale;  // h^2 / 36 (heat layout)
  const float* obs;  // observed elements (partial observation), or null
  // tracking mass M_s: the Q1 element masses M_e = (h/6)^d (x)_d [2 1; 1 2] of the observed
  // elements around the node; the plain mass without an observation mask
  template <typename F>
  IPM_D T track_f(const F& f, long long c) const {
    if (!obs) return mass_f(f, c);
    T acc = T(0);
    const int ne = dim == 3 ? 8 : 4;
    for (int e = 0; e < ne; ++e) {
      const int ea = e & 1, eb = (e >> 1) & 1, ec = (e >> 2) & 1;  // node's corner in the element
      const long long base = c - ea - (long long)eb * p - (long long)ec * pl;
      if (obs[base] == 0.f) continue;
      for (int q = 0; q < ne; ++q) {
        const int qa = q & 1, qb = (q >> 1) & 1, qc = (q >> 2) & 1;
        T w = (qa == ea ? T(2) : T(1)) * (qb == eb ? T(2) : T(1));
        if (dim == 3) w *= qc == ec ? T(2) : T(1);
        acc += w * f(base + qa + (long long)qb * p + (long long)qc * pl);
      }
    }
    return mscale * acc;
  }
  IPM_D T track(const T* __restrict__ x, long long c) const { return track_f(Ld<T>{x}, c); }
  template <typename F>
  IPM_D T mass_f(const F& f, long long c) const {
    return mscale * ((dim == 2 || heat) ? mass2_raw<T>(f, c, p) : mass3_raw<T>(f, c, p, pl));
  }
  // heat layout: the backward-Euler operator calL of Section 3.4 at time level k,
  // (M + tau K) x_k - M x_{k-1}, and its transpose (M + tau K) x_k - M x_{k+1}
  template <typename F>
  IPM_D T heat_L(const F& f, long long c, int dir) const {
    return m2scale * mass2_raw<T>(f, c, p) + tau * stiff2<T>(f, c, p) -
           m2scale * mass2_raw<T>(f, c + dir * pl, p);
  }
  template <typename F>
  IPM_D T stiff_f(const F& f, long long c) const {
    return dim == 2 ? stiff2<T>(f, c, p) : kscale * stiff3_raw<T>(f, c, p, pl);
  }
  IPM_D T mass(const T* __restrict__ x, long long c) const { return mass_f(Ld<T>{x}, c); }
  IPM_D T stiff(const T* __restrict__ x, long long c) const { return stiff_f(Ld<T>{x}, c); }
};

template <typename T>
inline Stencil<T> make_stencil(const GridDesc& g) {
  Stencil<T> s;
  s.dim = g.dim;
  s.p = g.pitch;
  s.pl = g.plane;
  s.mscale = g.dim == 2 ? T(g.h * g.h / 36.0) : T(g.h * g.h * g.h / 216.0);
  s.kscale = g.dim == 2 ? T(1) : T(g.h);
  s.heat = g.heat;
  s.tau = T(g.tau);
  s.m2scale = T(g.h * g.h / 36.0);
  if (g.heat) s.mscale = T(g.tau * g.h * g.h / 36.0);
  s.obs = g.obs;
  return s;
}

inline double mass_diag(const GridDesc& g) {  // (2h/3)^d; heat layout tau (2h/3)^2
  double t = 2.0 * g.h / 3.0;
  if (g.heat) return g.tau * t * t;
  return g.dim == 2 ? t * t : t * t * t;
}
inline double lumped_mass(const GridDesc& g) {  // h^d; heat layout tau h^2
  if (g.heat) return g.tau * g.h * g.h;
  return g.dim == 2 ? g.h * g.h : g.h * g.h * g.h;
}
inline double stiff_diag(const GridDesc& g) {  // 8/3 (2D) or 8h/3 (3D)
  return g.dim == 2 ? 8.0 / 3.0 : 8.0 * g.h / 3.0;
}

// ---------------------------------------------------------------------------
// Deterministic block reductions: fixed grid, fixed per-thread order, warp
// shuffles, then one partial per block; a second kernel sums the partials in
// block order. Results are bitwise reproducible run to run.
// ---------------------------------------------------------------------------
constexpr int kRedThreads = 256;
constexpr int kRedBlocks = 304;  // 2 x 152 SMs

template <typename T>
IPM_D T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}
template <typename T>
IPM_D T warp_min(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_down_sync(0xffffffffu, v, o));
  return v;
}

IPM_D int lin_tid() { return threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z); }
IPM_D int block_threads() { return blockDim.x * blockDim.y * blockDim.z; }
IPM_D long long lin_block() {
  return blockIdx.x + (long long)gridDim.x * (blockIdx.y + (long long)gridDim.y * blockIdx.z);
}
IPM_D long long num_blocks() { return (long long)gridDim.x * gridDim.y * gridDim.z; }

// Sum over the block (any shape, multiple of 32 threads); result valid in
// linear thread 0. `sh` needs (threads/32) entries. All threads must call.
template <typename T>
IPM_D T block_sum(T v, T* sh) {
  int t = lin_tid();
  int lane = t & 31, w = t >> 5, nw = block_threads() >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  T r = T(0);
  if (w == 0) {
    r = lane < nw ? sh[lane] : T(0);
    r = warp_sum(r);
  }
  __syncthreads();
  return r;
}
IPM_D double block_min(double v, double* sh) {
  int t = lin_tid();
  int lane = t & 31, w = t >> 5, nw = block_threads() >> 5;
  v = warp_min(v);
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  double r = 1e300;
  if (w == 0) {
    r = lane < nw ? sh[lane] : 1e300;
    r = warp_min(r);
  }
  __syncthreads();
  return r;
}

// ---------------------------------------------------------------------------
// Float-float (double-single) arithmetic: a value is the unevaluated sum h + l of two
// floats with |l| <= ulp(h) / 2. Error-free transformations: TwoSum (Knuth), FastTwoSum
// (Dekker, |a| >= |b|), and the exact product error of a fused multiply-add. Additions
// use the cheap form (one TwoSum plus the low parts), whose error is about
// 2^-46 (|a| + |b|). Used where FP64 arithmetic would bound a kernel: this GPU's FP64
// rate (and its FP64 <-> FP32 conversion rate) is about 1/70 of its FP32 rate. The _rn
// intrinsics keep the compiler from contracting the transformations into fused
// multiply-adds.
// ---------------------------------------------------------------------------
struct FF {
  float h, l;
};
IPM_D FF ff_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}
IPM_D FF ff_fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
IPM_D FF ff_add(FF a, FF b) {
  FF s = ff_two_sum(a.h, b.h);
  return ff_fast_two_sum(s.h, __fadd_rn(s.l, __fadd_rn(a.l, b.l)));
}
IPM_D FF ff_neg(FF a) { return {-a.h, -a.l}; }
IPM_D FF ff_mul(FF a, FF b) {
  const float p = __fmul_rn(a.h, b.h);
  const float e = fmaf(a.h, b.h, -p);
  return ff_fast_two_sum(p, __fadd_rn(e, fmaf(a.h, b.l, __fmul_rn(a.l, b.h))));
}
IPM_D double ff_to_double(FF a) { return (double)a.h + (double)a.l; }
IPM_D FF ff_from_double(double x) {
  const float h = __double2float_rn(x);
  return {h, __double2float_rn(x - (double)h)};
}

