// Fused geometric-multigrid kernels for the 2D Poisson operator L + diag(m).
//
// Same arithmetic as the per-sweep kernels of k_mg.cu (damped Jacobi with
// jinv = omega / (8/3 + m), residual, full-weighting restriction P^T, bilinear
// prolongation P), but each launch does many sweeps on a shared-memory tile:
//
//  k_mg2_pre_restrict  nu sweeps on a tile + halo (nu + 2), then the residual and
//                      the restriction onto the coarse nodes the tile owns;
//  k_mg2_prolong_post  x + P x_c on the tile + halo nu, then nu sweeps;
//  k_mg2_coarse        one CTA runs the whole V-cycle on all coarse levels (the
//                      caller picks them: up to 65^2 in FP32, 9^2 in FP64) in shared
//                      memory.
// The _rb forms of the first two (FP32, 5 sweeps) keep each thread's nodes in registers;
// k_cheb2_block / k_cheb2_rb do the same for blocks of Chebyshev steps.
//
// A V-cycle on a 1025^2 grid thus takes 2 launches per level above the coarse
// block plus one, instead of about 14 per level.
#include <cstdio>
#include <string>
#include <tuple>
#include <map>
#include <mutex>
#include <type_traits>

#include "kernels.h"

namespace {

constexpr int FTX = 64, FTY = 32;  // tile of fine nodes owned by one CTA (even sizes)

template <typename T>
IPM_D bool inside(int gx, int gy, int n) {
  return gx >= 1 && gx <= n - 2 && gy >= 1 && gy <= n - 2;
}

// A x at local index i of a shared tile with row stride SX (x = cur, m = sm)
template <typename T>
IPM_D T apply_A(const T* cur, int i, int SX, T mm) {
  T xc = cur[i];
  T box = (cur[i - SX - 1] + cur[i - SX] + cur[i - SX + 1]) + (cur[i - 1] + xc + cur[i + 1]) +
          (cur[i + SX - 1] + cur[i + SX] + cur[i + SX + 1]);
  return (T(3) * xc - box * T(1.0 / 3.0)) + mm * xc;
}

// nu damped-Jacobi sweeps on the shared tile; sweep s updates the region shrunk by s.
// Threads form a 32 x (blockDim / 32) grid over the region (no integer division).
template <typename T>
IPM_D void tile_sweeps(T*& cur, T*& nxt, const T* sb, const T* sm, const T* sj, int SX, int SY,
                       int X0, int Y0, int H, int n, int nu) {
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5, ny = blockDim.x >> 5;
  for (int s = 1; s <= nu; ++s) {
    for (int ly = s + ty; ly < SY - s; ly += ny) {
      const int gy = Y0 - H + ly;
      for (int lx = s + tx; lx < SX - s; lx += 32) {
        const int i = ly * SX + lx;
        T v = T(0);
        if (inside<T>(X0 - H + lx, gy, n)) {
          T xc = cur[i];
          T ax = apply_A(cur, i, SX, sm[i]);
          v = xc + sj[i] * (sb[i] - ax);
        }
        nxt[i] = v;
      }
    }
    __syncthreads();
    T* tmp = cur;
    cur = nxt;
    nxt = tmp;
  }
}

template <typename T, int TX, int TY>
__global__ void __launch_bounds__(512) k_mg2_pre_restrict(GridDesc g, GridDesc gc,
                                                          const T* __restrict__ xin,
                                                          T* __restrict__ xout,
                                                          const T* __restrict__ b,
                                                          const T* __restrict__ m,
                                                          T* __restrict__ bc, T omega, int nu,
                                                          int zero_init) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int H = nu + 2;
  const int SX = TX + 2 * H, SY = TY + 2 * H, S = SX * SY;
  T* s0 = reinterpret_cast<T*>(smem_raw);
  T* s1 = s0 + S;
  T* sb = s1 + S;
  T* sm = sb + S;
  T* sj = sm + S;
  const int X0 = blockIdx.x * TX, Y0 = blockIdx.y * TY;
  const int n = g.n, p = g.pitch;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5, ny = blockDim.x >> 5;
  for (int ly = ty; ly < SY; ly += ny) {
    const int gy = Y0 - H + ly;
    for (int lx = tx; lx < SX; lx += 32) {
      const int gx = X0 - H + lx, t = ly * SX + lx;
      bool in = inside<T>(gx, gy, n);
      long long c = (long long)gy * p + gx;
      T mm = in ? m[c] : T(0);
      s0[t] = (in && !zero_init) ? xin[c] : T(0);
      s1[t] = T(0);
      sb[t] = in ? b[c] : T(0);
      sm[t] = mm;
      sj[t] = omega / (T(8.0 / 3.0) + mm);
    }
  }
  __syncthreads();
  T* cur = s0;
  T* nxt = s1;
  tile_sweeps(cur, nxt, sb, sm, sj, SX, SY, X0, Y0, H, n, nu);
  // residual r = b - A x on the tile + halo 1 (into nxt)
  {
    const int lo = nu + 1;
    for (int ly = lo + ty; ly < SY - lo; ly += ny) {
      const int gy = Y0 - H + ly;
      for (int lx = lo + tx; lx < SX - lo; lx += 32) {
        const int i = ly * SX + lx;
        T r = T(0);
        if (inside<T>(X0 - H + lx, gy, n)) r = sb[i] - apply_A(cur, i, SX, sm[i]);
        nxt[i] = r;
      }
    }
  }
  __syncthreads();
  // full-weighting restriction onto the coarse nodes (2I, 2J) inside the tile
  const int nc = gc.n;
  for (int t = threadIdx.x; t < (TX / 2) * (TY / 2); t += blockDim.x) {
    int I = X0 / 2 + t % (TX / 2), J = Y0 / 2 + t / (TX / 2);
    if (I < 1 || I > nc - 2 || J < 1 || J > nc - 2) continue;
    int i = (2 * J - Y0 + H) * SX + (2 * I - X0 + H);
    T r0 = T(0.5) * nxt[i - SX - 1] + nxt[i - SX] + T(0.5) * nxt[i - SX + 1];
    T r1 = T(0.5) * nxt[i - 1] + nxt[i] + T(0.5) * nxt[i + 1];
    T r2 = T(0.5) * nxt[i + SX - 1] + nxt[i + SX] + T(0.5) * nxt[i + SX + 1];
    bc[(long long)J * gc.pitch + I] = T(0.5) * r0 + r1 + T(0.5) * r2;
  }
  for (int t = threadIdx.x; t < TX * TY; t += blockDim.x) {
    int gx = X0 + t % TX, gy = Y0 + t / TX;
    if (!inside<T>(gx, gy, n)) continue;
    xout[(long long)gy * p + gx] = cur[(gy - Y0 + H) * SX + (gx - X0 + H)];
  }
}

template <typename T>
IPM_D T prolong_at(const T* __restrict__ xc, int cp, int i, int j) {
  int i0 = i >> 1, j0 = j >> 1;
  int ni = (i & 1) ? 2 : 1, nj = (j & 1) ? 2 : 1;
  T wi = ni == 2 ? T(0.5) : T(1), wj = nj == 2 ? T(0.5) : T(1);
  T acc = T(0);
  for (int dj = 0; dj < nj; ++dj)
    for (int di = 0; di < ni; ++di) acc += xc[(long long)(j0 + dj) * cp + (i0 + di)];
  return wi * wj * T(1) * acc;
}

template <typename T, int TX, int TY>
__global__ void __launch_bounds__(512) k_mg2_prolong_post(GridDesc g, GridDesc gc,
                                                          const T* __restrict__ xin,
                                                          const T* __restrict__ xc,
                                                          T* __restrict__ xout,
                                                          const T* __restrict__ b,
                                                          const T* __restrict__ m, T omega,
                                                          int nu) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int H = nu;
  const int SX = TX + 2 * H, SY = TY + 2 * H, S = SX * SY;
  T* s0 = reinterpret_cast<T*>(smem_raw);
  T* s1 = s0 + S;
  T* sb = s1 + S;
  T* sm = sb + S;
  T* sj = sm + S;
  const int X0 = blockIdx.x * TX, Y0 = blockIdx.y * TY;
  const int n = g.n, p = g.pitch;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5, ny = blockDim.x >> 5;
  for (int ly = ty; ly < SY; ly += ny) {
    const int gy = Y0 - H + ly;
    for (int lx = tx; lx < SX; lx += 32) {
      const int gx = X0 - H + lx, t = ly * SX + lx;
      bool in = inside<T>(gx, gy, n);
      long long c = (long long)gy * p + gx;
      T mm = in ? m[c] : T(0);
      s0[t] = in ? xin[c] + prolong_at(xc, gc.pitch, gx, gy) : T(0);
      s1[t] = T(0);
      sb[t] = in ? b[c] : T(0);
      sm[t] = mm;
      sj[t] = omega / (T(8.0 / 3.0) + mm);
    }
  }
  __syncthreads();
  T* cur = s0;
  T* nxt = s1;
  tile_sweeps(cur, nxt, sb, sm, sj, SX, SY, X0, Y0, H, n, nu);
  for (int t = threadIdx.x; t < TX * TY; t += blockDim.x) {
    int gx = X0 + t % TX, gy = Y0 + t / TX;
    if (!inside<T>(gx, gy, n)) continue;
    xout[(long long)gy * p + gx] = cur[(gy - Y0 + H) * SX + (gx - X0 + H)];
  }
}

// ---------------------------------------------------------------------------
// Register-blocked FP32 tile kernels (same cycle pieces as the two kernels above, laid
// out for the shared-memory pipe; the stiffness stencil is evaluated on differences).
//
// Thread (lane, warp w) owns the tile nodes in columns 1 + lane + 32c (c < CX) and rows
// 1 + wK + r (r < K). The right-hand side, the diagonal m and the Jacobi weight of its
// nodes stay in registers for the whole launch; a sweep slides a three-row window down
// each owned column, so a node costs 3(K+2)/K shared loads and one store per sweep
// instead of twelve loads. Every sweep updates all nodes but the tile's outer ring: after
// sweep s the values within s nodes of the ring differ from the global sweep, and only
// nodes at least nu nodes inside (nu + 1 for the residual) are used afterwards.
// Tiles start at the first interior node, so ceil((n - 2) / T) tiles cover a direction.
// Nodes outside the domain carry zero weight and stay zero.
// ---------------------------------------------------------------------------
template <int TX, int TY, int H, int NW>
struct RBShape {
  static constexpr int SX = TX + 2 * H, SY = TY + 2 * H;
  static constexpr int CX = (SX - 2 + 31) / 32;
  static constexpr int K = (SY - 2 + NW - 1) / NW;
  static_assert(K * (NW - 1) < SY - 2, "every warp owns at least one row");
  static_assert(TX % 2 == 0 && TY % 2 == 0, "tiles own whole coarse cells");
  static constexpr size_t smem = 2 * (size_t)SX * SY * sizeof(float);
};

enum { kRBSweep = 0, kRBSweepOut = 1, kRBResidual = 2 };
constexpr int kRBSweeps = 5;  // sweeps per launch the register-blocked kernels are built for

// x into both tile buffers (ring by all threads, owned nodes by their owner) and the
// owned nodes' b, m, omega / diag into registers; load_x(gx, gy) gives x at an interior node
template <int TX, int TY, int H, int NW, typename LoadX>
IPM_D void rb_load(const GridDesc& g, int X0, int Y0, const float* __restrict__ b,
                   const float* __restrict__ m, float omega, const LoadX& load_x, float* cur,
                   float* nxt, float (&rb)[RBShape<TX, TY, H, NW>::CX][RBShape<TX, TY, H, NW>::K],
                   float (&rm)[RBShape<TX, TY, H, NW>::CX][RBShape<TX, TY, H, NW>::K],
                   float (&rj)[RBShape<TX, TY, H, NW>::CX][RBShape<TX, TY, H, NW>::K]) {
  using S = RBShape<TX, TY, H, NW>;
  constexpr int SX = S::SX, SY = S::SY;
  const int n = g.n, p = g.pitch;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int t = threadIdx.x; t < 2 * SX + 2 * (SY - 2); t += NW * 32) {
    int lx, ly;
    if (t < 2 * SX) {
      lx = t < SX ? t : t - SX;
      ly = t < SX ? 0 : SY - 1;
    } else {
      const int u = t - 2 * SX;
      ly = 1 + (u >> 1);
      lx = (u & 1) ? SX - 1 : 0;
    }
    const int gx = X0 - H + lx, gy = Y0 - H + ly;
    const float v = inside<float>(gx, gy, n) ? load_x(gx, gy) : 0.f;
    cur[ly * SX + lx] = v;
    nxt[ly * SX + lx] = v;
  }
#pragma unroll
  for (int c = 0; c < S::CX; ++c) {
    const int lx = 1 + lane + 32 * c;
#pragma unroll
    for (int r = 0; r < S::K; ++r) {
      const int ly = 1 + w * S::K + r;
      const int gx = X0 - H + lx, gy = Y0 - H + ly;
      float bb = 0.f, mm = 0.f, jj = 0.f;
      if (lx <= SX - 2 && ly <= SY - 2) {
        float xx = 0.f;
        if (inside<float>(gx, gy, n)) {
          const long long i = (long long)gy * p + gx;
          bb = b[i];
          mm = m[i];
          jj = omega / (float(8.0 / 3.0) + mm);
          xx = load_x(gx, gy);
        }
        cur[ly * SX + lx] = xx;
      }
      rb[c][r] = bb;
      rm[c][r] = mm;
      rj[c][r] = jj;
    }
  }
}

// one pass over the owned nodes: a Jacobi sweep into nxt (kRBSweep) or into xout for the
// nodes of the tile proper (kRBSweepOut), or the residual b - A x into nxt with x of the
// tile proper copied to xout (kRBResidual)
template <int MODE, int TX, int TY, int H, int NW>
IPM_D void rb_pass(const float* __restrict__ cur, float* __restrict__ nxt,
                   const float (&rb)[RBShape<TX, TY, H, NW>::CX][RBShape<TX, TY, H, NW>::K],
                   const float (&rm)[RBShape<TX, TY, H, NW>::CX][RBShape<TX, TY, H, NW>::K],
                   const float (&rj)[RBShape<TX, TY, H, NW>::CX][RBShape<TX, TY, H, NW>::K],
                   float* __restrict__ xout, const GridDesc& g, int X0, int Y0) {
  using S = RBShape<TX, TY, H, NW>;
  constexpr int SX = S::SX, SY = S::SY, K = S::K;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int ly0 = 1 + w * K;
#pragma unroll
  for (int c = 0; c < S::CX; ++c) {
    const int lx = 1 + lane + 32 * c;
    if (lx > SX - 2) continue;
    const float* col = cur + lx;
    const float* q = col + (ly0 - 1) * SX;
    float pl = q[-1], pc = q[0], pr = q[1];  // row above
    q = col + ly0 * SX;
    float cl = q[-1], xc = q[0], cr = q[1];  // this row
    const int gx = X0 - H + lx;
    const bool out_col = MODE != kRBSweep && lx >= H && lx < H + TX && gx <= g.n - 2;
#pragma unroll
    for (int r = 0; r < K; ++r) {
      const int ly = ly0 + r;
      if (K * NW > SY - 2 && ly > SY - 2) break;
      q = col + (ly + 1) * SX;
      const float nl = q[-1], xn = q[0], nr = q[1];  // row below
      // stiffness part as (1/3) sum over the 8 neighbours of (x_c - x_nb): the difference of
      // neighbouring values of a smooth field is exact in FP32 (Sterbenz), so this keeps
      // about 1/h more digits than 8 x_c - (sum of the 8) on fine grids
      const float s8 = (((xc - pl) + (xc - pc)) + ((xc - pr) + (xc - cl))) +
                       (((xc - cr) + (xc - nl)) + ((xc - xn) + (xc - nr)));
      const float ax = s8 * float(1.0 / 3.0) + rm[c][r] * xc;
      const int gy = Y0 - H + ly;
      const bool out = out_col && ly >= H && ly < H + TY && gy <= g.n - 2;
      if (MODE == kRBResidual) {
        nxt[ly * SX + lx] = rj[c][r] != 0.f ? rb[c][r] - ax : 0.f;
        if (out) xout[(long long)gy * g.pitch + gx] = xc;
      } else {
        const float v = xc + rj[c][r] * (rb[c][r] - ax);
        if (MODE == kRBSweep) nxt[ly * SX + lx] = v;
        else if (out) xout[(long long)gy * g.pitch + gx] = v;
      }
      pl = cl;
      pc = xc;
      pr = cr;
      cl = nl;
      xc = xn;
      cr = nr;
    }
  }
}

// pre-smoothing (NU sweeps from xin, or from zero), residual and full-weighting restriction
// of the tile with first interior node (X0, Y0); smem holds the two tile buffers
template <int TX, int TY, int NU, int NW>
IPM_D void pre_restrict_rb_tile(const GridDesc& g, const GridDesc& gc, const float* __restrict__ xin,
                                float* __restrict__ xout, const float* __restrict__ b,
                                const float* __restrict__ m, float* __restrict__ bc, float omega,
                                int zero_init, int X0, int Y0, unsigned char* smem_raw) {
  constexpr int H = NU + 2;
  using S = RBShape<TX, TY, H, NW>;
  constexpr int SX = S::SX;
  float* cur = reinterpret_cast<float*>(smem_raw);
  float* nxt = cur + SX * S::SY;
  const long long p = g.pitch;
  float rb[S::CX][S::K], rm[S::CX][S::K], rj[S::CX][S::K];
  auto load_x = [&](int gx, int gy) { return zero_init ? 0.f : xin[(long long)gy * p + gx]; };
  rb_load<TX, TY, H, NW>(g, X0, Y0, b, m, omega, load_x, cur, nxt, rb, rm, rj);
  __syncthreads();
#pragma unroll 1
  for (int s = 0; s < NU; ++s) {
    rb_pass<kRBSweep, TX, TY, H, NW>(cur, nxt, rb, rm, rj, nullptr, g, X0, Y0);
    __syncthreads();
    float* t = cur;
    cur = nxt;
    nxt = t;
  }
  rb_pass<kRBResidual, TX, TY, H, NW>(cur, nxt, rb, rm, rj, xout, g, X0, Y0);
  __syncthreads();
  // full weighting onto the coarse nodes I with 2I in [X0, X0 + TX) (X0 is odd)
  const int nc = gc.n;
  for (int t = threadIdx.x; t < (TX / 2) * (TY / 2); t += NW * 32) {
    const int I = (X0 + 1) / 2 + t % (TX / 2), J = (Y0 + 1) / 2 + t / (TX / 2);
    if (I > nc - 2 || J > nc - 2) continue;
    const int i = (2 * J - Y0 + H) * SX + (2 * I - X0 + H);
    const float r0 = 0.5f * nxt[i - SX - 1] + nxt[i - SX] + 0.5f * nxt[i - SX + 1];
    const float r1 = 0.5f * nxt[i - 1] + nxt[i] + 0.5f * nxt[i + 1];
    const float r2 = 0.5f * nxt[i + SX - 1] + nxt[i + SX] + 0.5f * nxt[i + SX + 1];
    bc[(long long)J * gc.pitch + I] = 0.5f * r0 + r1 + 0.5f * r2;
  }
}

template <int TX, int TY, int NU, int NW>
__global__ void __launch_bounds__(NW * 32) k_mg2_pre_restrict_rb(GridDesc g, GridDesc gc,
                                                                 const float* __restrict__ xin,
                                                                 float* __restrict__ xout,
                                                                 const float* __restrict__ b,
                                                                 const float* __restrict__ m,
                                                                 float* __restrict__ bc,
                                                                 float omega, int zero_init) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  pre_restrict_rb_tile<TX, TY, NU, NW>(g, gc, xin, xout, b, m, bc, omega, zero_init,
                                       1 + blockIdx.x * TX, 1 + blockIdx.y * TY, smem_raw);
}

// prolongation of the coarse correction xc onto xin and NU post-smoothing sweeps of the tile
// with first interior node (X0, Y0) into xout
template <int TX, int TY, int NU, int NW>
IPM_D void prolong_post_rb_tile(const GridDesc& g, const GridDesc& gc, const float* __restrict__ xin,
                                const float* __restrict__ xc, float* __restrict__ xout,
                                const float* __restrict__ b, const float* __restrict__ m,
                                float omega, int X0, int Y0, unsigned char* smem_raw) {
  constexpr int H = NU;
  using S = RBShape<TX, TY, H, NW>;
  float* cur = reinterpret_cast<float*>(smem_raw);
  float* nxt = cur + S::SX * S::SY;
  const long long p = g.pitch;
  const int cp = gc.pitch;
  float rb[S::CX][S::K], rm[S::CX][S::K], rj[S::CX][S::K];
  auto load_x = [&](int gx, int gy) {
    return xin[(long long)gy * p + gx] + prolong_at(xc, cp, gx, gy);
  };
  rb_load<TX, TY, H, NW>(g, X0, Y0, b, m, omega, load_x, cur, nxt, rb, rm, rj);
  __syncthreads();
#pragma unroll 1
  for (int s = 0; s < NU - 1; ++s) {
    rb_pass<kRBSweep, TX, TY, H, NW>(cur, nxt, rb, rm, rj, nullptr, g, X0, Y0);
    __syncthreads();
    float* t = cur;
    cur = nxt;
    nxt = t;
  }
  rb_pass<kRBSweepOut, TX, TY, H, NW>(cur, nxt, rb, rm, rj, xout, g, X0, Y0);
}

template <int TX, int TY, int NU, int NW>
__global__ void __launch_bounds__(NW * 32) k_mg2_prolong_post_rb(GridDesc g, GridDesc gc,
                                                                 const float* __restrict__ xin,
                                                                 const float* __restrict__ xc,
                                                                 float* __restrict__ xout,
                                                                 const float* __restrict__ b,
                                                                 const float* __restrict__ m,
                                                                 float omega) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  prolong_post_rb_tile<TX, TY, NU, NW>(g, gc, xin, xc, xout, b, m, omega, 1 + blockIdx.x * TX,
                                       1 + blockIdx.y * TY, smem_raw);
}

// ---------------------------------------------------------------------------
// One CTA, all coarse levels in shared memory (dense n x n per level).
// ---------------------------------------------------------------------------
// one damped-Jacobi sweep over the interior of an n x n level (threads as 32 x 32 grid)
template <typename T>
IPM_D void cta_sweep(const T* cur, T* nxt, const T* sb, const T* sm, const T* sj, int n, int zero) {
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5, ny = blockDim.x >> 5;
  for (int iy = 1 + ty; iy < n - 1; iy += ny)
    for (int ix = 1 + tx; ix < n - 1; ix += 32) {
      const int i = iy * n + ix;
      T xc = zero ? T(0) : cur[i];
      T ax = zero ? T(0) : apply_A(cur, i, n, sm[i]);
      nxt[i] = xc + sj[i] * (sb[i] - ax);
    }
}

// the V-cycle on the levels of cl for the Q1 stiffness + diag(m) (cl.general == 0): every
// level by the whole CTA, threads as a 32 x (blockDim / 32) grid
template <typename T>
IPM_D void coarse_cycle_box(const MGCoarse<T>& cl, const T* __restrict__ btop,
                            T* __restrict__ xtop, T omega, int nu_pre, int nu_post, int load_x,
                            unsigned char* smem_raw) {
  T* base = reinterpret_cast<T*>(smem_raw);
  // per-level size and offset of the six arrays (x0, x1, b, r, m, jinv) in a shared table,
  // and the current-iterate parity of every level as a register bit mask: indexing
  // per-thread arrays by the runtime level index would put them in local memory
  __shared__ int s_n[kMaxCoarse], s_off[kMaxCoarse];  // (per kernel, shared with coarse_cycle)
  __shared__ int s_pre[kMaxCoarse + 1];  // interior nodes of the levels before level l
  if (threadIdx.x == 0) {
    int off = 0, pre = 0;
    for (int l = 0; l < cl.nl; ++l) {
      s_n[l] = cl.n[l];
      s_off[l] = off;
      s_pre[l] = pre;
      off += 6 * cl.n[l] * cl.n[l];
      pre += (cl.n[l] - 2) * (cl.n[l] - 2);
    }
    s_pre[cl.nl] = pre;
  }
  __syncthreads();
  const int total = s_off[cl.nl - 1] + 6 * s_n[cl.nl - 1] * s_n[cl.nl - 1];
  auto arr = [&](int l, int a) { return base + s_off[l] + a * s_n[l] * s_n[l]; };
  enum { AX0 = 0, AX1 = 1, AB = 2, AR = 3, AM = 4, AJ = 5 };
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5, ny = blockDim.x >> 5;
  if constexpr (sizeof(T) == 4) {
    // FP32: the interior nodes of all levels as one flat range, kSlots per thread, so that
    // every global load of a thread is in flight at once (and behind the zeroing of the
    // shared arrays) instead of one level and one row at a time
    constexpr int kSlots = 6;
    const int nint = s_pre[cl.nl];
    for (int t0 = 0; t0 < nint; t0 += kSlots * (int)blockDim.x) {
      T vm[kSlots], vb[kSlots], vx[kSlots];
      int dst[kSlots], lev[kSlots];
#pragma unroll
      for (int k = 0; k < kSlots; ++k) {
        const int t = t0 + k * (int)blockDim.x + (int)threadIdx.x;
        lev[k] = -1;
        vm[k] = vb[k] = vx[k] = T(0);
        dst[k] = 0;
        if (t < nint) {
          int l = 0;
          while (t >= s_pre[l + 1]) ++l;
          const int w = s_n[l] - 2, r = t - s_pre[l];
          const int iy = 1 + r / w, ix = 1 + r - (iy - 1) * w;
          lev[k] = l;
          dst[k] = iy * s_n[l] + ix;
          vm[k] = cl.m[l][(long long)iy * cl.pitch[l] + ix];
          if (l == 0) {
            vb[k] = btop[(long long)iy * cl.pitch[0] + ix];
            if (load_x) vx[k] = xtop[(long long)iy * cl.pitch[0] + ix];
          }
        }
      }
      if (t0 == 0) {
        for (int t = threadIdx.x; t < total; t += blockDim.x) base[t] = T(0);
      }
      __syncthreads();
#pragma unroll
      for (int k = 0; k < kSlots; ++k) {
        const int l = lev[k];
        if (l < 0) continue;
        arr(l, AM)[dst[k]] = vm[k];
        arr(l, AJ)[dst[k]] = omega / (T(8.0 / 3.0) + vm[k]);
        if (l == 0) {
          arr(0, AB)[dst[k]] = vb[k];
          if (load_x) arr(0, AX0)[dst[k]] = vx[k];
        }
      }
    }
    if (nint == 0) {
      for (int t = threadIdx.x; t < total; t += blockDim.x) base[t] = T(0);
    }
  } else {
  // zero everything, then load b (top level) and m (all levels), interior entries
  for (int t = threadIdx.x; t < total; t += blockDim.x) base[t] = T(0);
  __syncthreads();
  for (int l = 0; l < cl.nl; ++l) {
    const int n = s_n[l];
    T* Ml = arr(l, AM);
    T* Jl = arr(l, AJ);
    const T* mg = cl.m[l];
    const long long pl = cl.pitch[l];
    for (int iy = 1 + ty; iy < n - 1; iy += ny)
      for (int ix = 1 + tx; ix < n - 1; ix += 32) {
        T mm = mg[(long long)iy * pl + ix];
        Ml[iy * n + ix] = mm;
        Jl[iy * n + ix] = omega / (T(8.0 / 3.0) + mm);
        if (l == 0) arr(0, AB)[iy * n + ix] = btop[(long long)iy * cl.pitch[0] + ix];
        if (l == 0 && load_x) arr(0, AX0)[iy * n + ix] = xtop[(long long)iy * cl.pitch[0] + ix];
      }
  }
  }
  __syncthreads();
  unsigned cur = 0;  // bit l: level l's current iterate is x1
  auto xcur = [&](int l) { return arr(l, ((cur >> l) & 1u) ? AX1 : AX0); };
  auto xnxt = [&](int l) { return arr(l, ((cur >> l) & 1u) ? AX0 : AX1); };
  const int L = cl.nl - 1;
  for (int l = 0; l < L; ++l) {
    const int n = s_n[l];
    const T* Bl = arr(l, AB);
    const T* Ml = arr(l, AM);
    const T* Jl = arr(l, AJ);
    T* Rl = arr(l, AR);
    for (int s = 0; s < nu_pre; ++s) {
      cta_sweep(xcur(l), xnxt(l), Bl, Ml, Jl, n, s == 0 && !(l == 0 && load_x));
      cur ^= 1u << l;
      __syncthreads();
    }
    {
      const T* c = xcur(l);
      for (int iy = 1 + ty; iy < n - 1; iy += ny)
        for (int ix = 1 + tx; ix < n - 1; ix += 32) {
          const int i = iy * n + ix;
          Rl[i] = Bl[i] - apply_A(c, i, n, Ml[i]);
        }
    }
    __syncthreads();
    {
      const int nc = s_n[l + 1];
      T* Bc = arr(l + 1, AB);
      for (int J = 1 + ty; J < nc - 1; J += ny)
        for (int I = 1 + tx; I < nc - 1; I += 32) {
          const int i = (2 * J) * n + 2 * I;
          const T* r = Rl;
          T r0 = T(0.5) * r[i - n - 1] + r[i - n] + T(0.5) * r[i - n + 1];
          T r1 = T(0.5) * r[i - 1] + r[i] + T(0.5) * r[i + 1];
          T r2 = T(0.5) * r[i + n - 1] + r[i + n] + T(0.5) * r[i + n + 1];
          Bc[J * nc + I] = T(0.5) * r0 + r1 + T(0.5) * r2;
        }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {  // coarsest grid: 3 nodes per direction, one unknown
    const int i = 1 * 3 + 1;
    arr(L, AX0)[i] = arr(L, AB)[i] / (T(8.0 / 3.0) + arr(L, AM)[i]);
  }
  cur &= ~(1u << L);
  __syncthreads();
  for (int l = L - 1; l >= 0; --l) {
    const int n = s_n[l], nc = s_n[l + 1];
    T* c = xcur(l);
    const T* xcs = xcur(l + 1);
    const bool wipe = nu_pre == 0 && !(l == 0 && load_x);  // x never written on this level
    for (int iy = 1 + ty; iy < n - 1; iy += ny)
      for (int ix = 1 + tx; ix < n - 1; ix += 32) {
        T base_v = wipe ? T(0) : c[iy * n + ix];
        c[iy * n + ix] = base_v + prolong_at(xcs, nc, ix, iy);
      }
    __syncthreads();
    const T* Bl = arr(l, AB);
    const T* Ml = arr(l, AM);
    const T* Jl = arr(l, AJ);
    for (int s = 0; s < nu_post; ++s) {
      cta_sweep(xcur(l), xnxt(l), Bl, Ml, Jl, n, 0);
      cur ^= 1u << l;
      __syncthreads();
    }
  }
  {
    const int n = s_n[0];
    const T* c = xcur(0);
    for (int iy = 1 + ty; iy < n - 1; iy += ny)
      for (int ix = 1 + tx; ix < n - 1; ix += 32) xtop[(long long)iy * cl.pitch[0] + ix] = c[iy * n + ix];
  }
}


// Work split of one level: the m = n - 2 interior columns times R row groups of K
// consecutive rows; thread t < m R owns column c = t % m, rows 1 + g K ... of group g = t / m.
// A thread reads its column and the two beside it once per row of its window (K + 2 rows)
// and forms the horizontal triple sums once, which the K outputs share.
constexpr int kCoarseK = 4;        // rows per thread at most (65^2: 63 columns x 16 groups of 4)
constexpr int kCoarseSmallN = 17;  // levels up to 17^2 run on the first 8 warps only
constexpr int kCoarseSmallThreads = 256;

struct Strip {
  int c, iy0, K;
  bool active;
};

IPM_D Strip strip_of(int n, int nthreads) {
  const int m = n - 2;
  int R = nthreads / m;
  if (R > m) R = m;
  if (R < 1) R = 1;
  Strip s;
  s.K = (m + R - 1) / R;
  const int t = threadIdx.x;
  s.active = t < m * R;
  s.c = t % m;
  s.iy0 = 1 + (t / m) * s.K;
  return s;
}

// mode 0: one damped-Jacobi sweep into out; mode 1: residual b - A x into out.
// zero: the iterate is zero (first sweep from x = 0).
// a constant symmetric 9-point stencil (centre, edge, corner weights)
template <typename T>
struct Stencil9 {
  bool on;
  T c0, ce, cc;
};

template <typename T>
IPM_D void strip_pass(const T* __restrict__ cur, T* __restrict__ out, const T* __restrict__ sb,
                      const T* __restrict__ sm, const T* __restrict__ sj, int n, const Strip& st,
                      int mode, bool zero, const Stencil9<T>& s9 = Stencil9<T>{false, T(0), T(0), T(0)}) {
  if (!st.active) return;
  if (s9.on && !zero) {
    // x_c, the horizontal pair sum l + r of each window row
    const int ix = st.c + 1;
    T lr[kCoarseK + 2], xm[kCoarseK + 2];
#pragma unroll
    for (int k = 0; k < kCoarseK + 2; ++k) {
      const int iy = st.iy0 - 1 + k;
      lr[k] = T(0);
      xm[k] = T(0);
      if (k < st.K + 2 && iy <= n - 1) {
        const T* r = cur + iy * n + ix;
        xm[k] = r[0];
        lr[k] = r[-1] + r[1];
      }
    }
#pragma unroll
    for (int k = 0; k < kCoarseK; ++k) {
      const int iy = st.iy0 + k;
      if (k < st.K && iy <= n - 2) {
        const int i = iy * n + ix;
        const T xc = xm[k + 1];
        const T edges = (lr[k + 1] + xm[k]) + xm[k + 2];
        const T corners = lr[k] + lr[k + 2];
        const T ax = (s9.c0 * xc + s9.ce * edges + s9.cc * corners) + sm[i] * xc;
        out[i] = mode == 0 ? xc + sj[i] * (sb[i] - ax) : sb[i] - ax;
      }
    }
    return;
  }
  const int ix = st.c + 1;
  if (zero) {
#pragma unroll
    for (int k = 0; k < kCoarseK; ++k) {
      const int iy = st.iy0 + k;
      if (k < st.K && iy <= n - 2) {
        const int i = iy * n + ix;
        out[i] = mode == 0 ? T(0) + sj[i] * (sb[i] - T(0)) : sb[i];
      }
    }
    return;
  }
  T h[kCoarseK + 2], xm[kCoarseK + 2];
#pragma unroll
  for (int k = 0; k < kCoarseK + 2; ++k) {
    const int iy = st.iy0 - 1 + k;
    h[k] = T(0);
    xm[k] = T(0);
    if (k < st.K + 2 && iy <= n - 1) {
      const T* r = cur + iy * n + ix;
      xm[k] = r[0];
      h[k] = (r[-1] + r[0]) + r[1];
    }
  }
#pragma unroll
  for (int k = 0; k < kCoarseK; ++k) {
    const int iy = st.iy0 + k;
    if (k < st.K && iy <= n - 2) {
      const int i = iy * n + ix;
      const T xc = xm[k + 1];
      const T box = (h[k] + h[k + 1]) + h[k + 2];
      const T ax = (T(3) * xc - box * T(1.0 / 3.0)) + sm[i] * xc;
      out[i] = mode == 0 ? xc + sj[i] * (sb[i] - ax) : sb[i] - ax;
    }
  }
}

// synchronisation of the threads working on a level: the whole CTA, or the first
// kCoarseSmallThreads threads (named barrier 1) on the small levels
IPM_D void coarse_sync(bool small) {
  if (small) asm volatile("bar.sync 1, %0;" ::"n"(kCoarseSmallThreads) : "memory");
  else __syncthreads();
}

// the V-cycle on the levels of cl, run by the whole CTA (any block size that is a multiple
// of 32, at least kCoarseSmallThreads, with no level above 65^2 for 1024 threads or above
// 33^2 for 256 threads); smem_raw holds mg2_coarse_smem(cl) bytes
template <typename T>
IPM_D void coarse_cycle(const MGCoarse<T>& cl, const T* __restrict__ btop, T* __restrict__ xtop,
                        T omega, int nu_pre, int nu_post, int load_x, unsigned char* smem_raw) {
  T* base = reinterpret_cast<T*>(smem_raw);
  // per-level size and offset of the six arrays (x0, x1, b, r, m, jinv) in a shared table,
  // and the current-iterate parity of every level as a register bit mask: indexing
  // per-thread arrays by the runtime level index would put them in local memory
  __shared__ int s_n[kMaxCoarse], s_off[kMaxCoarse];
  __shared__ unsigned s_cur;
  if (threadIdx.x == 0) {
    int off = 0;
    for (int l = 0; l < cl.nl; ++l) {
      s_n[l] = cl.n[l];
      s_off[l] = off;
      off += 6 * cl.n[l] * cl.n[l];
    }
  }
  __syncthreads();
  const int total = s_off[cl.nl - 1] + 6 * s_n[cl.nl - 1] * s_n[cl.nl - 1];
  auto arr = [&](int l, int a) { return base + s_off[l] + a * s_n[l] * s_n[l]; };
  enum { AX0 = 0, AX1 = 1, AB = 2, AR = 3, AM = 4, AJ = 5 };
  // zero everything, then load b (top level) and m (all levels), interior entries
  for (int t = threadIdx.x; t < total; t += blockDim.x) base[t] = T(0);
  __syncthreads();
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int l = 0; l < cl.nl; ++l) {
    const int n = s_n[l];
    T* Ml = arr(l, AM);
    T* Jl = arr(l, AJ);
    const T* mg = cl.m[l];
    const long long pl = cl.pitch[l];
    const int ny = blockDim.x >> 5;
    for (int iy = 1 + ty; iy < n - 1; iy += ny)
      for (int ix = 1 + tx; ix < n - 1; ix += 32) {
        T mm = mg[(long long)iy * pl + ix];
        Ml[iy * n + ix] = mm;
        Jl[iy * n + ix] = omega / ((cl.general ? cl.c0[l] : T(8.0 / 3.0)) + mm);
        if (l == 0) arr(0, AB)[iy * n + ix] = btop[(long long)iy * cl.pitch[0] + ix];
        if (l == 0 && load_x) arr(0, AX0)[iy * n + ix] = xtop[(long long)iy * cl.pitch[0] + ix];
      }
  }
  __syncthreads();
  unsigned cur = 0;  // bit l: level l's current iterate is x1
  auto xcur = [&](int l) { return arr(l, ((cur >> l) & 1u) ? AX1 : AX0); };
  auto xnxt = [&](int l) { return arr(l, ((cur >> l) & 1u) ? AX0 : AX1); };
  const int L = cl.nl - 1;
  int ls = 0;  // first small level
  while (ls < L && s_n[ls] > kCoarseSmallN) ++ls;

  auto s9of = [&](int l) { return Stencil9<T>{cl.general != 0, cl.c0[l], cl.ce[l], cl.cc[l]}; };
  // pre-smoothing, residual and full-weighting restriction of level l
  auto descend = [&](int l, bool small) {
    const int n = s_n[l];
    const Stencil9<T> s9 = s9of(l);
    const int nthr = small ? kCoarseSmallThreads : (int)blockDim.x;
    const Strip st = strip_of(n, nthr);
    const T* Bl = arr(l, AB);
    const T* Ml = arr(l, AM);
    const T* Jl = arr(l, AJ);
    T* Rl = arr(l, AR);
    for (int s = 0; s < nu_pre; ++s) {
      strip_pass(xcur(l), xnxt(l), Bl, Ml, Jl, n, st, 0, s == 0 && !(l == 0 && load_x), s9);
      cur ^= 1u << l;
      coarse_sync(small);
    }
    strip_pass(xcur(l), Rl, Bl, Ml, Jl, n, st, 1, false, s9);
    coarse_sync(small);
    const int nc = s_n[l + 1];
    T* Bc = arr(l + 1, AB);
    const int ny = nthr >> 5;
    for (int J = 1 + ty; J < nc - 1; J += ny)
      for (int I = 1 + tx; I < nc - 1; I += 32) {
        const int i = (2 * J) * n + 2 * I;
        const T* r = Rl;
        T r0 = T(0.5) * r[i - n - 1] + r[i - n] + T(0.5) * r[i - n + 1];
        T r1 = T(0.5) * r[i - 1] + r[i] + T(0.5) * r[i + 1];
        T r2 = T(0.5) * r[i + n - 1] + r[i + n] + T(0.5) * r[i + n + 1];
        Bc[J * nc + I] = T(0.5) * r0 + r1 + T(0.5) * r2;
      }
    coarse_sync(small);
  };
  // prolongation of the coarse correction and post-smoothing of level l
  auto ascend = [&](int l, bool small) {
    const int n = s_n[l], nc = s_n[l + 1];
    const int nthr = small ? kCoarseSmallThreads : (int)blockDim.x;
    const Strip st = strip_of(n, nthr);
    T* c = xcur(l);
    const T* xcs = xcur(l + 1);
    const bool wipe = nu_pre == 0 && !(l == 0 && load_x);  // x never written on this level
    if (st.active) {
      const int ix = st.c + 1;
#pragma unroll
      for (int k = 0; k < kCoarseK; ++k) {
        const int iy = st.iy0 + k;
        if (k < st.K && iy <= n - 2) {
          T base_v = wipe ? T(0) : c[iy * n + ix];
          c[iy * n + ix] = base_v + prolong_at(xcs, nc, ix, iy);
        }
      }
    }
    coarse_sync(small);
    const T* Bl = arr(l, AB);
    const T* Ml = arr(l, AM);
    const T* Jl = arr(l, AJ);
    const Stencil9<T> s9 = s9of(l);
    for (int s = 0; s < nu_post; ++s) {
      strip_pass(xcur(l), xnxt(l), Bl, Ml, Jl, n, st, 0, false, s9);
      cur ^= 1u << l;
      coarse_sync(small);
    }
  };

  for (int l = 0; l < ls; ++l) descend(l, false);
  if (threadIdx.x < kCoarseSmallThreads) {
    for (int l = ls; l < L; ++l) descend(l, true);
    if (threadIdx.x == 0) {  // coarsest grid: 3 nodes per direction, one unknown
      const int i = 1 * 3 + 1;
      arr(L, AX0)[i] = arr(L, AB)[i] / ((cl.general ? cl.c0[L] : T(8.0 / 3.0)) + arr(L, AM)[i]);
    }
    cur &= ~(1u << L);
    coarse_sync(true);
    for (int l = L - 1; l >= ls; --l) ascend(l, true);
    if (threadIdx.x == 0) s_cur = cur;
  }
  __syncthreads();
  cur = s_cur;  // the small levels' parities, set by the threads that ran them
  for (int l = ls - 1; l >= 0; --l) ascend(l, false);
  {
    const int n = s_n[0];
    const T* c = xcur(0);
    const int ny = blockDim.x >> 5;
    for (int iy = 1 + ty; iy < n - 1; iy += ny)
      for (int ix = 1 + tx; ix < n - 1; ix += 32) xtop[(long long)iy * cl.pitch[0] + ix] = c[iy * n + ix];
  }
}

template <typename T>
__global__ void __launch_bounds__(1024) k_mg2_coarse(MGCoarse<T> cl, const T* __restrict__ btop,
                                                     T* __restrict__ xtop, T omega, int nu_pre,
                                                     int nu_post, int load_x) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  coarse_cycle_box<T>(cl, btop, xtop, omega, nu_pre, nu_post, load_x, smem_raw);
}

// the same cycle for a constant 9-point stencil per level (cl.general == 1)
template <typename T>
__global__ void __launch_bounds__(1024) k_mg2_coarse9(MGCoarse<T> cl, const T* __restrict__ btop,
                                                      T* __restrict__ xtop, T omega, int nu_pre,
                                                      int nu_post, int load_x) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  coarse_cycle<T>(cl, btop, xtop, omega, nu_pre, nu_post, load_x, smem_raw);
}

// ---------------------------------------------------------------------------
// Persistent V-cycle below the finest level (cooperative launch, grid-wide barriers).
// ---------------------------------------------------------------------------
constexpr int kMidPreTX = 20, kMidPreTY = 32, kMidPostT = 24, kMidNW = 8;
constexpr long long kBarrierSpins = 1ll << 22;  // a few seconds at most with the sleeps

// All blocks of the grid meet here (the blocks are co-resident: cooperative launch).
// Thread 0 of each block arrives on a counter; the last one resets it and advances the
// generation, the others wait for the generation to change. A wait beyond the spin budget
// sets bar->timeout and returns false (as does any wait once a timeout is recorded).
IPM_D bool grid_barrier(GridBarrier* bar, unsigned nblocks) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* vgen = &bar->gen;
    volatile int* vto = &bar->timeout;
    const unsigned g0 = *vgen;
    __threadfence();
    int ok = 1;
    if (atomicAdd(&bar->count, 1u) == nblocks - 1) {
      atomicExch(&bar->count, 0u);
      __threadfence();
      atomicAdd(&bar->gen, 1u);
    } else {
      long long spins = 0;
      while (*vgen == g0) {
        if (*vto || ++spins > kBarrierSpins) {
          atomicExch(&bar->timeout, 1);
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

__global__ void __launch_bounds__(kMidNW * 32) k_mg2_mid_cycle(MidCycle mc, GridBarrier* bar,
                                                               float omega) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const unsigned nb = gridDim.x;
  bool ok = true;
  for (int l = 0; l < mc.nt && ok; ++l) {
    const GridDesc& g = mc.g[l];
    const int tx = (g.n - 2 + kMidPreTX - 1) / kMidPreTX, ty = (g.n - 2 + kMidPreTY - 1) / kMidPreTY;
    for (int t = blockIdx.x; t < tx * ty; t += gridDim.x) {
      __syncthreads();  // the block's previous tile is done with the shared buffers
      pre_restrict_rb_tile<kMidPreTX, kMidPreTY, kRBSweeps, kMidNW>(
          g, mc.g[l + 1], nullptr, mc.xb[l], mc.b[l], mc.m[l], mc.bnext[l], omega, 1,
          1 + (t % tx) * kMidPreTX, 1 + (t / tx) * kMidPreTY, smem_raw);
    }
    ok = grid_barrier(bar, nb);
  }
  if (ok) {
    if (blockIdx.x == 0)
      coarse_cycle_box<float>(mc.cl, mc.bnext[mc.nt - 1], mc.xcoarse, omega, kRBSweeps,
                              kRBSweeps, 0, smem_raw);
    ok = grid_barrier(bar, nb);
  }
  for (int l = mc.nt - 1; l >= 0 && ok; --l) {
    const GridDesc& g = mc.g[l];
    const float* xc = l == mc.nt - 1 ? mc.xcoarse : mc.xa[l + 1];
    const int tx = (g.n - 2 + kMidPostT - 1) / kMidPostT;
    for (int t = blockIdx.x; t < tx * tx; t += gridDim.x) {
      __syncthreads();
      prolong_post_rb_tile<kMidPostT, kMidPostT, kRBSweeps, kMidNW>(
          g, mc.g[l + 1], mc.xb[l], xc, mc.xa[l], mc.b[l], mc.m[l], omega,
          1 + (t % tx) * kMidPostT, 1 + (t / tx) * kMidPostT, smem_raw);
    }
    ok = grid_barrier(bar, nb);
  }
  // a barrier that gave up leaves a non-finite value in the cycle's output, which the
  // Krylov iteration reports as a breakdown
  if (blockIdx.x == 0 && threadIdx.x == 0 && *(volatile int*)&bar->timeout)
    mc.xa[0][mc.g[0].pitch + 1] = __int_as_float(0x7fc00000);
}

template <typename T>
size_t tile_smem(int halo, int tx, int ty) {
  return 5 * (size_t)(tx + 2 * halo) * (ty + 2 * halo) * sizeof(T);
}

// raise a kernel's dynamic shared memory limit when a launch needs more than the default.
// The attribute is per device, so the raised limit is remembered per (kernel, device); it
// only grows, under a lock (solvers on several host threads launch concurrently). A failed
// cudaFuncSetAttribute is not remembered: the launch that follows then fails, and the
// solver's next error check reports IPM_ECUDA.
std::mutex g_smem_attr_mu;
std::map<std::pair<const void*, int>, size_t> g_smem_attr_set;
void ensure_smem_attr(const void* fn, size_t bytes) {
  if (bytes <= 48 * 1024) return;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return;
  std::lock_guard<std::mutex> lk(g_smem_attr_mu);
  size_t& set_to = g_smem_attr_set[{fn, dev}];
  if (bytes > set_to &&
      cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) ==
          cudaSuccess)
    set_to = bytes;
}

}  // namespace

template <typename T>
size_t mg2_coarse_smem(const MGCoarse<T>& cl) {
  size_t s = 0;
  for (int l = 0; l < cl.nl; ++l) s += 6 * (size_t)cl.n[l] * cl.n[l];
  return s * sizeof(T);
}

// large levels: 64 x 32 tiles, 512 threads; smaller levels: 32 x 16 tiles, 256 threads
// (shorter per-CTA latency and more CTAs in flight where there are few tiles)
template <typename T, int TX, int TY>
void pre_restrict_tiles(const GridDesc& g, const GridDesc& gc, const T* xin, T* xout, const T* b,
                        const T* m, T* bc, double omega, int nu, int zero_init, int threads,
                        cudaStream_t s) {
  size_t sm = tile_smem<T>(nu + 2, TX, TY);
  ensure_smem_attr((const void*)k_mg2_pre_restrict<T, TX, TY>, sm);
  dim3 grid((g.n + TX - 1) / TX, (g.n + TY - 1) / TY);
  count_launches(1);
  k_mg2_pre_restrict<T, TX, TY><<<grid, threads, sm, s>>>(g, gc, xin, xout, b, m, bc, (T)omega, nu,
                                                          zero_init);
}

template <int TX, int TY, int NW>
void pre_restrict_rb(const GridDesc& g, const GridDesc& gc, const float* xin, float* xout,
                     const float* b, const float* m, float* bc, double omega, int zero_init,
                     cudaStream_t s) {
  constexpr int NU = kRBSweeps;
  const size_t sm = RBShape<TX, TY, NU + 2, NW>::smem;
  ensure_smem_attr((const void*)k_mg2_pre_restrict_rb<TX, TY, NU, NW>, sm);
  dim3 grid((g.n - 2 + TX - 1) / TX, (g.n - 2 + TY - 1) / TY);
  count_launches(1);
  k_mg2_pre_restrict_rb<TX, TY, NU, NW><<<grid, NW * 32, sm, s>>>(g, gc, xin, xout, b, m, bc,
                                                                 (float)omega, zero_init);
}

template <int TX, int TY, int NW>
void prolong_post_rb(const GridDesc& g, const GridDesc& gc, const float* xin, const float* xc,
                     float* xout, const float* b, const float* m, double omega, cudaStream_t s) {
  constexpr int NU = kRBSweeps;
  const size_t sm = RBShape<TX, TY, NU, NW>::smem;
  ensure_smem_attr((const void*)k_mg2_prolong_post_rb<TX, TY, NU, NW>, sm);
  dim3 grid((g.n - 2 + TX - 1) / TX, (g.n - 2 + TY - 1) / TY);
  count_launches(1);
  k_mg2_prolong_post_rb<TX, TY, NU, NW><<<grid, NW * 32, sm, s>>>(g, gc, xin, xc, xout, b, m,
                                                                 (float)omega);
}

// ---------------------------------------------------------------------------
// Tile-shape autotuning of the register-blocked FP32 kernels. Candidate shapes keep the
// halo'd tile width a whole number of 32-lane column groups (TX + 12 for the 7-node halo
// of pre-smoothing, TX + 8 for the 5-node halo of post-smoothing); every shape computes
// each node with the same arithmetic, so the choice changes timing only. The choice per
// (kernel, grid size, device) is made once per process by timing every candidate on the
// caller's buffers (mg2_autotune); until then, and for sizes never tuned, the fixed rule
// of the timing sweep that chose the defaults applies.
// ---------------------------------------------------------------------------
namespace {
constexpr int kPreShapes = 7, kPostShapes = 7;
const char* const kPreShapeNames[kPreShapes] = {"52x52/16w", "20x32/8w", "52x32/8w", "52x24/8w",
                                                "20x64/8w", "20x18/8w", "20x36/16w"};
const char* const kPostShapeNames[kPostShapes] = {"56x32/8w", "24x24/8w", "56x56/16w", "24x48/8w",
                                                  "56x24/8w", "24x16/8w", "24x40/16w"};

void pre_rb_shape(int c, const GridDesc& g, const GridDesc& gc, const float* xin, float* xout,
                  const float* b, const float* m, float* bc, double omega, int zero_init,
                  cudaStream_t s) {
  switch (c) {
    case 0: pre_restrict_rb<52, 52, 16>(g, gc, xin, xout, b, m, bc, omega, zero_init, s); break;
    case 1: pre_restrict_rb<20, 32, 8>(g, gc, xin, xout, b, m, bc, omega, zero_init, s); break;
    case 2: pre_restrict_rb<52, 32, 8>(g, gc, xin, xout, b, m, bc, omega, zero_init, s); break;
    case 3: pre_restrict_rb<52, 24, 8>(g, gc, xin, xout, b, m, bc, omega, zero_init, s); break;
    case 4: pre_restrict_rb<20, 64, 8>(g, gc, xin, xout, b, m, bc, omega, zero_init, s); break;
    case 5: pre_restrict_rb<20, 18, 8>(g, gc, xin, xout, b, m, bc, omega, zero_init, s); break;
    default: pre_restrict_rb<20, 36, 16>(g, gc, xin, xout, b, m, bc, omega, zero_init, s); break;
  }
}

void post_rb_shape(int c, const GridDesc& g, const GridDesc& gc, const float* xin, const float* xc,
                   float* xout, const float* b, const float* m, double omega, cudaStream_t s) {
  switch (c) {
    case 0: prolong_post_rb<56, 32, 8>(g, gc, xin, xc, xout, b, m, omega, s); break;
    case 1: prolong_post_rb<24, 24, 8>(g, gc, xin, xc, xout, b, m, omega, s); break;
    case 2: prolong_post_rb<56, 56, 16>(g, gc, xin, xc, xout, b, m, omega, s); break;
    case 3: prolong_post_rb<24, 48, 8>(g, gc, xin, xc, xout, b, m, omega, s); break;
    case 4: prolong_post_rb<56, 24, 8>(g, gc, xin, xc, xout, b, m, omega, s); break;
    case 5: prolong_post_rb<24, 16, 8>(g, gc, xin, xc, xout, b, m, omega, s); break;
    default: prolong_post_rb<24, 40, 16>(g, gc, xin, xc, xout, b, m, omega, s); break;
  }
}

struct TuneEntry {
  int shape;
  double us;  // average launch time of the chosen shape
};
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int>, TuneEntry> g_tuned;  // (kernel, n, device) -> choice

int tuned_shape(int kernel, int n) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return -1;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto it = g_tuned.find({kernel, n, dev});
  return it == g_tuned.end() ? -1 : it->second.shape;
}
}  // namespace

template <typename T>
void launch_mg2_pre_restrict(const GridDesc& g, const GridDesc& gc, const T* xin, T* xout,
                             const T* b, const T* m, T* bc, double omega, int nu, int zero_init,
                             cudaStream_t s) {
  if constexpr (std::is_same<T, float>::value) {
    if (nu == kRBSweeps) {
      int c = tuned_shape(0, g.n);
      if (c < 0) c = g.n > 513 ? 0 : 1;  // fixed rule from a timing sweep on GB300
      pre_rb_shape(c, g, gc, xin, xout, b, m, bc, omega, zero_init, s);
      return;
    }
  }
  if (g.n >= 513)
    pre_restrict_tiles<T, 64, 32>(g, gc, xin, xout, b, m, bc, omega, nu, zero_init, 512, s);
  else
    pre_restrict_tiles<T, 32, 16>(g, gc, xin, xout, b, m, bc, omega, nu, zero_init, 256, s);
}

template <typename T, int TX, int TY>
void prolong_post_tiles(const GridDesc& g, const GridDesc& gc, const T* xin, const T* xc, T* xout,
                        const T* b, const T* m, double omega, int nu, int threads,
                        cudaStream_t s) {
  size_t sm = tile_smem<T>(nu, TX, TY);
  ensure_smem_attr((const void*)k_mg2_prolong_post<T, TX, TY>, sm);
  dim3 grid((g.n + TX - 1) / TX, (g.n + TY - 1) / TY);
  count_launches(1);
  k_mg2_prolong_post<T, TX, TY><<<grid, threads, sm, s>>>(g, gc, xin, xc, xout, b, m, (T)omega,
                                                          nu);
}

template <typename T>
void launch_mg2_prolong_post(const GridDesc& g, const GridDesc& gc, const T* xin, const T* xc,
                             T* xout, const T* b, const T* m, double omega, int nu,
                             cudaStream_t s) {
  if constexpr (std::is_same<T, float>::value) {
    if (nu == kRBSweeps) {
      int c = tuned_shape(1, g.n);
      if (c < 0) c = g.n > 513 ? 0 : 1;
      post_rb_shape(c, g, gc, xin, xc, xout, b, m, omega, s);
      return;
    }
  }
  if (g.n >= 513) prolong_post_tiles<T, 64, 32>(g, gc, xin, xc, xout, b, m, omega, nu, 512, s);
  else prolong_post_tiles<T, 32, 16>(g, gc, xin, xc, xout, b, m, omega, nu, 256, s);
}

template <typename T>
void launch_mg2_coarse(const MGCoarse<T>& cl, const T* btop, T* xtop, double omega, int nu_pre,
                       int nu_post, int load_x, cudaStream_t s) {
  size_t sm = mg2_coarse_smem(cl);
  count_launches(1);
  if (cl.general) {
    ensure_smem_attr((const void*)k_mg2_coarse9<T>, sm);
    k_mg2_coarse9<T><<<1, 1024, sm, s>>>(cl, btop, xtop, (T)omega, nu_pre, nu_post, load_x);
  } else {
    ensure_smem_attr((const void*)k_mg2_coarse<T>, sm);
    k_mg2_coarse<T><<<1, 1024, sm, s>>>(cl, btop, xtop, (T)omega, nu_pre, nu_post, load_x);
  }
}

bool mg2_is_tuned(int n) { return tuned_shape(0, n) >= 0 && tuned_shape(1, n) >= 0; }

int mg2_autotune(const GridDesc& g, const GridDesc& gc, float* xa, float* xb, const float* b,
                 const float* m, float* bc, const float* xc, double omega, cudaStream_t s) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 1;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return 1;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return 1;
  }
  constexpr int kReps = 16;
  int rc = 0;
  for (int kernel = 0; kernel < 2 && rc == 0; ++kernel) {
    const int ncand = kernel == 0 ? kPreShapes : kPostShapes;
    int best = -1;
    float best_ms = 0.f;
    for (int c = 0; c < ncand && rc == 0; ++c) {
      auto run = [&] {
        if (kernel == 0) pre_rb_shape(c, g, gc, xa, xb, b, m, bc, omega, 0, s);
        else post_rb_shape(c, g, gc, xb, xc, xa, b, m, omega, s);
      };
      run();  // first launch: attributes, module load
      cudaEventRecord(e0, s);
      for (int r = 0; r < kReps; ++r) run();
      cudaEventRecord(e1, s);
      float ms = 0.f;
      if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
        rc = 1;
        break;
      }
      count_launches(-(kReps + 1));  // tuning launches are not the solver's work
      if (best < 0 || ms < best_ms) {
        best = c;
        best_ms = ms;
      }
    }
    if (rc == 0 && best >= 0) {
      std::lock_guard<std::mutex> lk(g_tune_mu);
      g_tuned[{kernel, g.n, dev}] = TuneEntry{best, 1000.0 * best_ms / kReps};
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaGetLastError();
  return rc;
}

int mg2_tune_set(int kernel, int n, int shape) {
  if (kernel < 0 || kernel > 1 || n < 3) return 1;
  if (shape >= (kernel == 0 ? kPreShapes : kPostShapes)) return 1;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 1;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  if (shape < 0) g_tuned.erase({kernel, n, dev});
  else g_tuned[{kernel, n, dev}] = TuneEntry{shape, 0.0};
  return 0;
}

int mg2_tune_report(char* buf, size_t len) {
  std::string out;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  for (const auto& kv : g_tuned) {
    const int kernel = std::get<0>(kv.first), n = std::get<1>(kv.first);
    char line[160];
    std::snprintf(line, sizeof(line), "%s n=%d dev=%d: %s %.2f us\n",
                  kernel == 0 ? "pre_restrict" : "prolong_post", n, std::get<2>(kv.first),
                  kernel == 0 ? kPreShapeNames[kv.second.shape] : kPostShapeNames[kv.second.shape],
                  kv.second.us);
    out += line;
  }
  if (buf && len > 0) {
    std::snprintf(buf, len, "%s", out.c_str());
  }
  return (int)out.size();
}

#define IPM_MG2_INST(T)                                                                           \
  template size_t mg2_coarse_smem<T>(const MGCoarse<T>&);                                        \
  template void launch_mg2_pre_restrict<T>(const GridDesc&, const GridDesc&, const T*, T*,       \
                                           const T*, const T*, T*, double, int, int,             \
                                           cudaStream_t);                                         \
  template void launch_mg2_prolong_post<T>(const GridDesc&, const GridDesc&, const T*, const T*, \
                                           T*, const T*, const T*, double, int, cudaStream_t);   \
  template void launch_mg2_coarse<T>(const MGCoarse<T>&, const T*, T*, double, int, int, int,     \
                                     cudaStream_t);
IPM_MG2_INST(float)
IPM_MG2_INST(double)

namespace {
size_t mid_cycle_smem(const MidCycle& mc) {
  size_t sm = RBShape<kMidPreTX, kMidPreTY, kRBSweeps + 2, kMidNW>::smem;
  sm = std::max(sm, RBShape<kMidPostT, kMidPostT, kRBSweeps, kMidNW>::smem);
  return std::max(sm, mg2_coarse_smem<float>(mc.cl));
}
}  // namespace

int mg2_mid_blocks(const MidCycle& mc) {
  int dev = 0, coop = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess || !coop ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  const size_t sm = mid_cycle_smem(mc);
  ensure_smem_attr((const void*)k_mg2_mid_cycle, sm);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_mg2_mid_cycle, kMidNW * 32, sm) !=
          cudaSuccess ||
      per_sm < 1) {
    cudaGetLastError();
    return 0;
  }
  int tiles = 1;
  for (int l = 0; l < mc.nt; ++l) {
    const int m = mc.g[l].n - 2;
    const int pre = ((m + kMidPreTX - 1) / kMidPreTX) * ((m + kMidPreTY - 1) / kMidPreTY);
    const int post = ((m + kMidPostT - 1) / kMidPostT) * ((m + kMidPostT - 1) / kMidPostT);
    tiles = std::max(tiles, std::max(pre, post));
  }
  return std::min(tiles, per_sm * sms);
}

void launch_mg2_mid_cycle(const MidCycle& mc, GridBarrier* bar, double omega, int blocks,
                          cudaStream_t s) {
  const size_t sm = mid_cycle_smem(mc);
  ensure_smem_attr((const void*)k_mg2_mid_cycle, sm);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(blocks);
  cfg.blockDim = dim3(kMidNW * 32);
  cfg.dynamicSmemBytes = sm;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  count_launches(1);
  cudaLaunchKernelEx(&cfg, k_mg2_mid_cycle, mc, bar, (float)omega);
}

// ---------------------------------------------------------------------------
// Chebyshev semi-iteration for (M + Theta_y) x = b, temporally blocked (2D):
// `ns` steps per launch on a 64x32 tile with halo ns, both iterates in shared
// memory. Step k: x_{k+1} = x_k + (w_k - 1)(x_k - x_{k-1}) + w_k g J^{-1}(b - A x_k),
// J = D_M + Theta_y, g = 1/theta; `first` starts from x_0 = 0, x_1 = g J^{-1} b.
// ---------------------------------------------------------------------------
namespace {

template <typename T, typename Ti, typename To>
__global__ void __launch_bounds__(512) k_cheb2_block(GridDesc g, ChebSteps cs, const Ti* __restrict__ b,
                                                     const T* __restrict__ thy, const T* xc_in,
                                                     const T* xp_in, T* xc_out, T* xp_out,
                                                     To* final_out, int first) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int H = cs.ns;
  const int SX = FTX + 2 * H, SY = FTY + 2 * H, S = SX * SY;
  T* sa = reinterpret_cast<T*>(smem_raw);
  T* sbuf = sa + S;
  T* sc = sbuf + S;
  T* sb = sc + S;
  T* st = sb + S;
  T* sinv = st + S;  // 1 / (D_M + Theta_y)
  const int X0 = blockIdx.x * FTX, Y0 = blockIdx.y * FTY;
  const int n = g.n, p = g.pitch;
  const T dM = (T)cs.dM, gam = (T)cs.gamma, ms = (T)cs.mscale;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5, ny = blockDim.x >> 5;
  T* prev = sa;
  T* cur = sbuf;
  T* nxt = sc;
  for (int ly = ty; ly < SY; ly += ny) {
    const int gy = Y0 - H + ly;
    for (int lx = tx; lx < SX; lx += 32) {
      const int gx = X0 - H + lx, t = ly * SX + lx;
      bool in = inside<T>(gx, gy, n);
      long long c = (long long)gy * p + gx;
      T bb = in ? (T)b[c] : T(0);
      T th = in ? thy[c] : T(0);
      T iv = T(1) / (dM + th);
      sb[t] = bb;
      st[t] = th;
      sinv[t] = iv;
      if (first) {
        prev[t] = T(0);
        cur[t] = in ? gam * bb * iv : T(0);
      } else {
        prev[t] = in ? xp_in[c] : T(0);
        cur[t] = in ? xc_in[c] : T(0);
      }
      nxt[t] = T(0);
    }
  }
  __syncthreads();
  for (int s = 1; s <= cs.ns; ++s) {
    const T om = (T)cs.omega[s - 1];
    const T og = om * gam;
    for (int ly = s + ty; ly < SY - s; ly += ny) {
      const int gy = Y0 - H + ly;
      for (int lx = s + tx; lx < SX - s; lx += 32) {
        const int i = ly * SX + lx;
        T v = T(0);
        if (inside<T>(X0 - H + lx, gy, n)) {
          T x = cur[i];
          T r0 = cur[i - SX - 1] + T(4) * cur[i - SX] + cur[i - SX + 1];
          T r1 = cur[i - 1] + T(4) * x + cur[i + 1];
          T r2 = cur[i + SX - 1] + T(4) * cur[i + SX] + cur[i + SX + 1];
          T ax = ms * (r0 + T(4) * r1 + r2) + st[i] * x;
          v = x + (om - T(1)) * (x - prev[i]) + og * (sb[i] - ax) * sinv[i];
        }
        nxt[i] = v;
      }
    }
    __syncthreads();
    T* tmp = prev;
    prev = cur;
    cur = nxt;
    nxt = tmp;
  }
  for (int t = threadIdx.x; t < FTX * FTY; t += blockDim.x) {
    int gx = X0 + t % FTX, gy = Y0 + t / FTX;
    if (!inside<T>(gx, gy, n)) continue;
    int i = (gy - Y0 + H) * SX + (gx - X0 + H);
    long long c = (long long)gy * p + gx;
    if (final_out) {
      final_out[c] = (To)cur[i];
    } else {
      xc_out[c] = cur[i];
      xp_out[c] = prev[i];
    }
  }
}

// Register-blocked FP32 form of k_cheb2_block (same recurrence and arithmetic): the
// owner of a node keeps its b, Theta_y, 1 / (D_M + Theta_y) and previous iterate in
// registers, the current iterate is exchanged through shared memory. Nodes outside the
// domain carry a zero inverse diagonal and stay zero.
template <int TX, int TY, int NS, int NW, typename Ti>
__global__ void __launch_bounds__(NW * 32) k_cheb2_rb(GridDesc g, ChebSteps cs,
                                                      const Ti* __restrict__ b,
                                                      const float* __restrict__ thy,
                                                      const float* xc_in, const float* xp_in,
                                                      float* xc_out, float* xp_out,
                                                      double* final_out, float* final32,
                                                      int first) {
  constexpr int H = NS;
  using S = RBShape<TX, TY, H, NW>;
  constexpr int SX = S::SX, SY = S::SY, CX = S::CX, K = S::K;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* cur = reinterpret_cast<float*>(smem_raw);
  float* nxt = cur + SX * SY;
  const int X0 = 1 + blockIdx.x * TX, Y0 = 1 + blockIdx.y * TY;
  const int n = g.n;
  const long long p = g.pitch;
  const float dM = (float)cs.dM, gam = (float)cs.gamma, ms = (float)cs.mscale;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int t = threadIdx.x; t < 2 * SX + 2 * (SY - 2); t += NW * 32) {
    int lx, ly;
    if (t < 2 * SX) {
      lx = t < SX ? t : t - SX;
      ly = t < SX ? 0 : SY - 1;
    } else {
      const int u = t - 2 * SX;
      ly = 1 + (u >> 1);
      lx = (u & 1) ? SX - 1 : 0;
    }
    const int gx = X0 - H + lx, gy = Y0 - H + ly;
    float v = 0.f;
    if (inside<float>(gx, gy, n)) {
      const long long c = (long long)gy * p + gx;
      if (first) v = gam * (float)b[c] * (1.0f / (dM + thy[c]));
      else v = xc_in[c];
    }
    cur[ly * SX + lx] = v;
    nxt[ly * SX + lx] = v;
  }
  float rb[CX][K], rt[CX][K], ri[CX][K], rp[CX][K];
#pragma unroll
  for (int c = 0; c < CX; ++c) {
    const int lx = 1 + lane + 32 * c;
#pragma unroll
    for (int r = 0; r < K; ++r) {
      const int ly = 1 + w * K + r;
      const int gx = X0 - H + lx, gy = Y0 - H + ly;
      float bb = 0.f, th = 0.f, iv = 0.f, xp = 0.f;
      if (lx <= SX - 2 && ly <= SY - 2) {
        float x = 0.f;
        if (inside<float>(gx, gy, n)) {
          const long long i = (long long)gy * p + gx;
          bb = (float)b[i];
          th = thy[i];
          iv = 1.0f / (dM + th);
          if (first) {
            x = gam * bb * iv;
          } else {
            x = xc_in[i];
            xp = xp_in[i];
          }
        }
        cur[ly * SX + lx] = x;
      }
      rb[c][r] = bb;
      rt[c][r] = th;
      ri[c][r] = iv;
      rp[c][r] = xp;
    }
  }
  __syncthreads();
  const int ly0 = 1 + w * K;
#pragma unroll
  for (int s = 1; s <= NS; ++s) {
    const float om = (float)cs.omega[s - 1];
    const float og = om * gam;
    const bool last = s == NS;
#pragma unroll
    for (int c = 0; c < CX; ++c) {
      const int lx = 1 + lane + 32 * c;
      if (lx > SX - 2) continue;
      const float* col = cur + lx;
      const float* q = col + (ly0 - 1) * SX;
      float hp = (q[-1] + 4.0f * q[0]) + q[1];
      q = col + ly0 * SX;
      float xc = q[0];
      float hc = (q[-1] + 4.0f * xc) + q[1];
      const int gx = X0 - H + lx;
      const bool out_col = lx >= H && lx < H + TX && gx <= n - 2;
#pragma unroll
      for (int r = 0; r < K; ++r) {
        const int ly = ly0 + r;
        if (K * NW > SY - 2 && ly > SY - 2) break;
        q = col + (ly + 1) * SX;
        const float xn = q[0];
        const float hn = (q[-1] + 4.0f * xn) + q[1];
        const float ax = ms * ((hp + 4.0f * hc) + hn) + rt[c][r] * xc;
        const float v = xc + (om - 1.0f) * (xc - rp[c][r]) + og * (rb[c][r] - ax) * ri[c][r];
        if (last) {
          const int gy = Y0 - H + ly;
          if (out_col && ly >= H && ly < H + TY && gy <= n - 2) {
            const long long i = (long long)gy * p + gx;
            if (final_out) {
              final_out[i] = (double)v;
              if (final32) final32[i] = v;
            } else {
              xc_out[i] = v;
              xp_out[i] = xc;
            }
          }
        } else {
          nxt[ly * SX + lx] = v;
        }
        rp[c][r] = xc;
        hp = hc;
        hc = hn;
        xc = xn;
      }
    }
    if (!last) {
      __syncthreads();
      float* t = cur;
      cur = nxt;
      nxt = t;
    }
  }
}

template <int TX, int TY, int NS, int NW, typename Ti>
void cheb2_rb(const GridDesc& g, const ChebSteps& cs, const Ti* b, const float* thy,
              const float* xc_in, const float* xp_in, float* xc_out, float* xp_out,
              double* final_out, float* final32, int first, cudaStream_t s) {
  const size_t sm = RBShape<TX, TY, NS, NW>::smem;
  ensure_smem_attr((const void*)k_cheb2_rb<TX, TY, NS, NW, Ti>, sm);
  dim3 grid((g.n - 2 + TX - 1) / TX, (g.n - 2 + TY - 1) / TY);
  count_launches(1);
  k_cheb2_rb<TX, TY, NS, NW, Ti><<<grid, NW * 32, sm, s>>>(g, cs, b, thy, xc_in, xp_in, xc_out,
                                                            xp_out, final_out, final32, first);
}

// FP32 iterates: register-blocked kernels for blocks of 4 or 5 steps
template <int NS, typename Ti>
void cheb2_rb_dispatch(const GridDesc& g, const ChebSteps& cs, const Ti* b, const float* thy,
                       const float* xc_in, const float* xp_in, float* xc_out, float* xp_out,
                       double* final_out, float* final32, int first, cudaStream_t s) {
  if (g.n > 513)
    cheb2_rb<56, 32, NS, 8, Ti>(g, cs, b, thy, xc_in, xp_in, xc_out, xp_out, final_out, final32,
                                first, s);
  else
    cheb2_rb<24, 24, NS, 8, Ti>(g, cs, b, thy, xc_in, xp_in, xc_out, xp_out, final_out, final32,
                                first, s);
}

}  // namespace

template <typename T, typename Ti, typename To>
void launch_cheb2_block(const GridDesc& g, const ChebSteps& cs, const Ti* b, const T* thy,
                        const T* xc_in, const T* xp_in, T* xc_out, T* xp_out, To* final_out,
                        int first, cudaStream_t s) {
  if constexpr (std::is_same<T, float>::value && std::is_same<Ti, double>::value &&
                std::is_same<To, double>::value) {
    if (cs.ns == 5) {
      cheb2_rb_dispatch<5, double>(g, cs, b, thy, xc_in, xp_in, xc_out, xp_out, final_out,
                                   nullptr, first, s);
      return;
    }
    if (cs.ns == 4) {
      cheb2_rb_dispatch<4, double>(g, cs, b, thy, xc_in, xp_in, xc_out, xp_out, final_out,
                                   nullptr, first, s);
      return;
    }
  }
  size_t sm = 6 * (size_t)(FTX + 2 * cs.ns) * (FTY + 2 * cs.ns) * sizeof(T);
  ensure_smem_attr((const void*)k_cheb2_block<T, Ti, To>, sm);
  dim3 grid((g.n + FTX - 1) / FTX, (g.n + FTY - 1) / FTY);
  count_launches(1);
  k_cheb2_block<T, Ti, To><<<grid, 512, sm, s>>>(g, cs, b, thy, xc_in, xp_in, xc_out, xp_out,
                                                 final_out, first);
}

// FP32 right-hand side (the high parts of a float-float vector) and an FP32 copy of the
// final iterate; blocks of 4 or 5 steps (false otherwise: nothing launched)
bool launch_cheb2_rb_f32(const GridDesc& g, const ChebSteps& cs, const float* b, const float* thy,
                         const float* xc_in, const float* xp_in, float* xc_out, float* xp_out,
                         double* final_out, float* final32, int first, cudaStream_t s) {
  if (cs.ns == 5)
    cheb2_rb_dispatch<5, float>(g, cs, b, thy, xc_in, xp_in, xc_out, xp_out, final_out, final32,
                                first, s);
  else if (cs.ns == 4)
    cheb2_rb_dispatch<4, float>(g, cs, b, thy, xc_in, xp_in, xc_out, xp_out, final_out, final32,
                                first, s);
  else
    return false;
  return true;
}

#define IPM_CHEB2_INST(T, Ti, To)                                                              \
  template void launch_cheb2_block<T, Ti, To>(const GridDesc&, const ChebSteps&, const Ti*,   \
                                              const T*, const T*, const T*, T*, T*, To*, int, \
                                              cudaStream_t);
IPM_CHEB2_INST(float, double, double)
IPM_CHEB2_INST(double, double, double)
