// Fused geometric-multigrid kernels for the 2D Poisson operator L + diag(m).
//
// Same arithmetic as the per-sweep kernels of k_mg.cu (damped Jacobi with
// jinv = omega / (8/3 + m), residual, full-weighting restriction P^T, bilinear
// prolongation P), but each launch does many sweeps on a shared-memory tile:
//
//  k_mg2_pre_restrict  nu sweeps on a 64x32 tile + halo (nu + 2), then the residual
//                      and the restriction onto the coarse nodes the tile owns;
//  k_mg2_prolong_post  x + P x_c on the tile + halo nu, then nu sweeps;
//  k_mg2_coarse        one CTA runs the whole V-cycle on all levels at or below
//                      65^2 (FP32) / 33^2 (FP64) in shared memory.
//
// A V-cycle on a 1025^2 grid thus takes 2 launches per level above the coarse
// block plus one, instead of about 14 per level.
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

template <typename T>
__global__ void __launch_bounds__(1024) k_mg2_coarse(MGCoarse<T> cl, const T* __restrict__ btop,
                                                     T* __restrict__ xtop, T omega, int nu_pre,
                                                     int nu_post, int load_x) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* base = reinterpret_cast<T*>(smem_raw);
  T* X0[kMaxCoarse];
  T* X1[kMaxCoarse];
  T* B[kMaxCoarse];
  T* R[kMaxCoarse];
  T* Mm[kMaxCoarse];
  T* Jv[kMaxCoarse];
  int off = 0;
  for (int l = 0; l < cl.nl; ++l) {
    int s = cl.n[l] * cl.n[l];
    X0[l] = base + off;
    X1[l] = X0[l] + s;
    B[l] = X1[l] + s;
    R[l] = B[l] + s;
    Mm[l] = R[l] + s;
    Jv[l] = Mm[l] + s;
    off += 6 * s;
  }
  // zero everything, then load b (top level) and m (all levels), interior entries
  for (int t = threadIdx.x; t < off; t += blockDim.x) base[t] = T(0);
  __syncthreads();
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5, ny = blockDim.x >> 5;
  for (int l = 0; l < cl.nl; ++l) {
    int n = cl.n[l];
    for (int iy = 1 + ty; iy < n - 1; iy += ny)
      for (int ix = 1 + tx; ix < n - 1; ix += 32) {
        T mm = cl.m[l][(long long)iy * cl.pitch[l] + ix];
        Mm[l][iy * n + ix] = mm;
        Jv[l][iy * n + ix] = omega / (T(8.0 / 3.0) + mm);
        if (l == 0) B[0][iy * n + ix] = btop[(long long)iy * cl.pitch[0] + ix];
        if (l == 0 && load_x) X0[0][iy * n + ix] = xtop[(long long)iy * cl.pitch[0] + ix];
      }
  }
  __syncthreads();
  int cur[kMaxCoarse];
  for (int l = 0; l < cl.nl; ++l) cur[l] = 0;
  const int L = cl.nl - 1;
  for (int l = 0; l < L; ++l) {
    int n = cl.n[l];
    for (int s = 0; s < nu_pre; ++s) {
      T* c = cur[l] ? X1[l] : X0[l];
      T* nx = cur[l] ? X0[l] : X1[l];
      cta_sweep(c, nx, B[l], Mm[l], Jv[l], n, s == 0 && !(l == 0 && load_x));
      cur[l] ^= 1;
      __syncthreads();
    }
    {
      T* c = cur[l] ? X1[l] : X0[l];
      for (int iy = 1 + ty; iy < n - 1; iy += ny)
        for (int ix = 1 + tx; ix < n - 1; ix += 32) {
          const int i = iy * n + ix;
          R[l][i] = B[l][i] - apply_A(c, i, n, Mm[l][i]);
        }
    }
    __syncthreads();
    {
      int nc = cl.n[l + 1];
      for (int J = 1 + ty; J < nc - 1; J += ny)
        for (int I = 1 + tx; I < nc - 1; I += 32) {
          int i = (2 * J) * n + 2 * I;
          const T* r = R[l];
          T r0 = T(0.5) * r[i - n - 1] + r[i - n] + T(0.5) * r[i - n + 1];
          T r1 = T(0.5) * r[i - 1] + r[i] + T(0.5) * r[i + 1];
          T r2 = T(0.5) * r[i + n - 1] + r[i + n] + T(0.5) * r[i + n + 1];
          B[l + 1][J * nc + I] = T(0.5) * r0 + r1 + T(0.5) * r2;
        }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {  // coarsest grid: 3 nodes per direction, one unknown
    int i = 1 * 3 + 1;
    X0[L][i] = B[L][i] / (T(8.0 / 3.0) + Mm[L][i]);
    cur[L] = 0;
  }
  __syncthreads();
  for (int l = L - 1; l >= 0; --l) {
    int n = cl.n[l], nc = cl.n[l + 1];
    T* c = cur[l] ? X1[l] : X0[l];
    const T* xcs = cur[l + 1] ? X1[l + 1] : X0[l + 1];
    const bool wipe = nu_pre == 0 && !(l == 0 && load_x);  // x never written on this level
    for (int iy = 1 + ty; iy < n - 1; iy += ny)
      for (int ix = 1 + tx; ix < n - 1; ix += 32) {
        T base_v = wipe ? T(0) : c[iy * n + ix];
        c[iy * n + ix] = base_v + prolong_at(xcs, nc, ix, iy);
      }
    __syncthreads();
    for (int s = 0; s < nu_post; ++s) {
      T* cc = cur[l] ? X1[l] : X0[l];
      T* nx = cur[l] ? X0[l] : X1[l];
      cta_sweep(cc, nx, B[l], Mm[l], Jv[l], n, 0);
      cur[l] ^= 1;
      __syncthreads();
    }
  }
  {
    int n = cl.n[0];
    const T* c = cur[0] ? X1[0] : X0[0];
    for (int iy = 1 + ty; iy < n - 1; iy += ny)
      for (int ix = 1 + tx; ix < n - 1; ix += 32) xtop[(long long)iy * cl.pitch[0] + ix] = c[iy * n + ix];
  }
}

template <typename T>
size_t tile_smem(int halo, int tx, int ty) {
  return 5 * (size_t)(tx + 2 * halo) * (ty + 2 * halo) * sizeof(T);
}

// raise a kernel's dynamic shared memory limit when a launch needs more than the default
void ensure_smem_attr(const void* fn, size_t bytes, size_t& set_to) {
  if (bytes > 48 * 1024 && bytes > set_to) {
    cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    set_to = bytes;
  }
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
  static size_t set_to = 0;
  size_t sm = tile_smem<T>(nu + 2, TX, TY);
  ensure_smem_attr((const void*)k_mg2_pre_restrict<T, TX, TY>, sm, set_to);
  dim3 grid((g.n + TX - 1) / TX, (g.n + TY - 1) / TY);
  count_launches(1);
  k_mg2_pre_restrict<T, TX, TY><<<grid, threads, sm, s>>>(g, gc, xin, xout, b, m, bc, (T)omega, nu,
                                                          zero_init);
}

template <typename T>
void launch_mg2_pre_restrict(const GridDesc& g, const GridDesc& gc, const T* xin, T* xout,
                             const T* b, const T* m, T* bc, double omega, int nu, int zero_init,
                             cudaStream_t s) {
  if (g.n >= 513)
    pre_restrict_tiles<T, 64, 32>(g, gc, xin, xout, b, m, bc, omega, nu, zero_init, 512, s);
  else
    pre_restrict_tiles<T, 32, 16>(g, gc, xin, xout, b, m, bc, omega, nu, zero_init, 256, s);
}

template <typename T, int TX, int TY>
void prolong_post_tiles(const GridDesc& g, const GridDesc& gc, const T* xin, const T* xc, T* xout,
                        const T* b, const T* m, double omega, int nu, int threads,
                        cudaStream_t s) {
  static size_t set_to = 0;
  size_t sm = tile_smem<T>(nu, TX, TY);
  ensure_smem_attr((const void*)k_mg2_prolong_post<T, TX, TY>, sm, set_to);
  dim3 grid((g.n + TX - 1) / TX, (g.n + TY - 1) / TY);
  count_launches(1);
  k_mg2_prolong_post<T, TX, TY><<<grid, threads, sm, s>>>(g, gc, xin, xc, xout, b, m, (T)omega,
                                                          nu);
}

template <typename T>
void launch_mg2_prolong_post(const GridDesc& g, const GridDesc& gc, const T* xin, const T* xc,
                             T* xout, const T* b, const T* m, double omega, int nu,
                             cudaStream_t s) {
  if (g.n >= 513) prolong_post_tiles<T, 64, 32>(g, gc, xin, xc, xout, b, m, omega, nu, 512, s);
  else prolong_post_tiles<T, 32, 16>(g, gc, xin, xc, xout, b, m, omega, nu, 256, s);
}

template <typename T>
void launch_mg2_coarse(const MGCoarse<T>& cl, const T* btop, T* xtop, double omega, int nu_pre,
                       int nu_post, int load_x, cudaStream_t s) {
  static size_t set_to = 0;
  size_t sm = mg2_coarse_smem(cl);
  ensure_smem_attr((const void*)k_mg2_coarse<T>, sm, set_to);
  count_launches(1);
  k_mg2_coarse<T><<<1, 1024, sm, s>>>(cl, btop, xtop, (T)omega, nu_pre, nu_post, load_x);
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

}  // namespace

template <typename T, typename Ti, typename To>
void launch_cheb2_block(const GridDesc& g, const ChebSteps& cs, const Ti* b, const T* thy,
                        const T* xc_in, const T* xp_in, T* xc_out, T* xp_out, To* final_out,
                        int first, cudaStream_t s) {
  static size_t set_to = 0;
  size_t sm = 6 * (size_t)(FTX + 2 * cs.ns) * (FTY + 2 * cs.ns) * sizeof(T);
  ensure_smem_attr((const void*)k_cheb2_block<T, Ti, To>, sm, set_to);
  dim3 grid((g.n + FTX - 1) / FTX, (g.n + FTY - 1) / FTY);
  count_launches(1);
  k_cheb2_block<T, Ti, To><<<grid, 512, sm, s>>>(g, cs, b, thy, xc_in, xp_in, xc_out, xp_out,
                                                 final_out, first);
}

#define IPM_CHEB2_INST(T, Ti, To)                                                              \
  template void launch_cheb2_block<T, Ti, To>(const GridDesc&, const ChebSteps&, const Ti*,   \
                                              const T*, const T*, const T*, T*, T*, To*, int, \
                                              cudaStream_t);
IPM_CHEB2_INST(float, double, double)
IPM_CHEB2_INST(double, double, double)
