// Krylov vector kernels over contiguous blocks of fields (FP64).
//
// Reductions run on a fixed grid (kRedBlocks x kRedThreads) with a fixed
// per-thread traversal order, so that every dot product is bitwise
// reproducible; partial sums are then added in block order.
#include "kernels.h"
#include <atomic>

// process-wide total, and the calling thread's share (graph capture counts the launches it
// records from the thread's share, which other host threads' solvers do not change)
static std::atomic<long long> g_launches{0};
static thread_local long long t_launches = 0;
void count_launches(long long n) {
  g_launches.fetch_add(n, std::memory_order_relaxed);
  t_launches += n;
}
long long launches_total() { return g_launches.load(std::memory_order_relaxed); }
long long launches_thread() { return t_launches; }

namespace {

constexpr int kMaxDots = 8;

__global__ void k_multidot(const double* __restrict__ V, long long stride, int nv,
                           const double* __restrict__ w, long long len, double* __restrict__ part) {
  __shared__ double sh[32];
  double acc[kMaxDots];
#pragma unroll
  for (int q = 0; q < kMaxDots; ++q) acc[q] = 0.0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < len;
       e += (long long)gridDim.x * blockDim.x) {
    double we = w[e];
#pragma unroll
    for (int q = 0; q < kMaxDots; ++q)
      if (q < nv) acc[q] += V[q * stride + e] * we;
  }
  for (int q = 0; q < nv; ++q) {
    double r = block_sum(acc[q], sh);
    if (threadIdx.x == 0) part[(long long)blockIdx.x * kMaxDots + q] = r;
  }
}

__global__ void k_reduce_dots(const double* __restrict__ part, int nblocks, int nv,
                              double* __restrict__ out) {
  __shared__ double sh[32];
  int q = blockIdx.x;
  double acc = 0.0;
  for (int r = threadIdx.x; r < nblocks; r += blockDim.x) acc += part[(long long)r * kMaxDots + q];
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0) out[q] = acc;
}

// w += sign * sum_q coef[q] V_q
__global__ void k_axpy_multi(double* __restrict__ w, const double* __restrict__ V, long long stride,
                             int nv, const double* __restrict__ coef, double sign, long long len) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < len;
       e += (long long)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int q = 0; q < nv; ++q) acc += coef[q] * V[q * stride + e];
    w[e] += sign * acc;
  }
}

__global__ void k_axpby(double* y, const double* x, double a, double b,
                        long long len) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < len;
       e += (long long)gridDim.x * blockDim.x)
    y[e] = b == 0.0 ? a * x[e] : a * x[e] + b * y[e];  // b = 0 never reads y
}

int vec_blocks(long long len) {
  long long b = (len + 255) / 256;
  return (int)(b < 4 * kRedBlocks ? b : 4 * kRedBlocks);
}

}  // namespace

void launch_multidot(const double* V, long long stride, int nv, const double* w, long long len,
                     double* part, double* out, cudaStream_t s) {
  for (int q0 = 0; q0 < nv; q0 += kMaxDots) {
    int m = nv - q0 < kMaxDots ? nv - q0 : kMaxDots;
    count_launches(1);
    k_multidot<<<kRedBlocks, kRedThreads, 0, s>>>(V + q0 * stride, stride, m, w, len, part);
    count_launches(1);
    k_reduce_dots<<<m, 256, 0, s>>>(part, kRedBlocks, m, out + q0);
  }
}
void launch_axpy_multi(double* w, const double* V, long long stride, int nv, const double* coef,
                       double sign, long long len, cudaStream_t s) {
  count_launches(1);
  k_axpy_multi<<<vec_blocks(len), 256, 0, s>>>(w, V, stride, nv, coef, sign, len);
}
void launch_axpby(double* y, const double* x, double a, double b, long long len, cudaStream_t s) {
  count_launches(1);
  k_axpby<<<vec_blocks(len), 256, 0, s>>>(y, x, a, b, len);
}
void launch_dot(const double* a, const double* b, long long len, double* part, double* out,
                cudaStream_t s) {
  launch_multidot(a, 0, 1, b, len, part, out, s);
}

namespace {
__global__ void k_lincomb3(double* __restrict__ y, double a, const double* __restrict__ x1, double b,
                           const double* __restrict__ x2, double c, const double* __restrict__ x3,
                           long long len) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < len;
       e += (long long)gridDim.x * blockDim.x) {
    double v = a * x1[e];
    if (x2) v += b * x2[e];
    if (x3) v += c * x3[e];
    y[e] = v;
  }
}
}  // namespace

namespace {
// y = x / sqrt(s[0])  (normalisation by a device-side squared norm)
__global__ void k_scale_rsqrt(double* y, const double* x, const double* __restrict__ s,
                              long long len) {
  double f = 1.0 / sqrt(s[0]);
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < len;
       e += (long long)gridDim.x * blockDim.x)
    y[e] = x[e] * f;
}
}  // namespace

void launch_scale_rsqrt(double* y, const double* x, const double* s, long long len,
                        cudaStream_t st) {
  count_launches(1);
  k_scale_rsqrt<<<vec_blocks(len), 256, 0, st>>>(y, x, s, len);
}

void launch_lincomb3(double* y, double a, const double* x1, double b, const double* x2, double c,
                     const double* x3, long long len, cudaStream_t s) {
  count_launches(1);
  k_lincomb3<<<vec_blocks(len), 256, 0, s>>>(y, a, x1, b, x2, c, x3, len);
}

// ---------------------------------------------------------------------------
// Float-float Krylov vectors: a 4-field vector of `len` entries stored as its high parts
// (len floats) followed by its low parts (len floats), in the memory of an FP64 vector.
// Products and sums run in float-float arithmetic; block partial sums are written in
// FP64 and reduced in block order as in the FP64 kernels (bitwise reproducible).
// ---------------------------------------------------------------------------
namespace {

IPM_D FF ff_at(const float* v, long long len, long long e) { return {v[e], v[len + e]}; }

IPM_D FF warp_sum_ff(FF v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    FF u{__shfl_down_sync(0xffffffffu, v.h, o), __shfl_down_sync(0xffffffffu, v.l, o)};
    v = ff_add(v, u);
  }
  return v;
}

// sum over the block, valid in thread 0 (blockDim.x a multiple of 32, <= 1024)
IPM_D FF block_sum_ff(FF v, FF* sh) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = warp_sum_ff(v);
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  FF r{0.f, 0.f};
  if (w == 0) {
    if (lane < nw) r = sh[lane];
    r = warp_sum_ff(r);
  }
  __syncthreads();
  return r;
}

// Dot products in float-float: each term's exact product error (fused multiply-add) and
// the running sum's TwoSum error go to a separate compensation sum (the scheme of
// Ogita, Rump and Oishi's Dot2, with float-float inputs). Four consecutive entries per
// thread and step (16-byte loads; len is a multiple of 4 and every vector 16-byte aligned).
IPM_D void dot2_step(float& sum, float& cmp, float ah, float al, float bh, float bl) {
  const float p = __fmul_rn(ah, bh);
  const float pe = fmaf(ah, bh, -p);
  const FF s = ff_two_sum(sum, p);
  sum = s.h;
  cmp = __fadd_rn(cmp, __fadd_rn(__fadd_rn(pe, s.l), fmaf(ah, bl, __fmul_rn(al, bh))));
}

__global__ void k_multidot_ff(const float* __restrict__ V, long long stride, int nv,
                              const float* __restrict__ w, long long len,
                              double* __restrict__ part) {
  __shared__ FF sh[32];
  float sum[kMaxDots], cmp[kMaxDots];
#pragma unroll
  for (int q = 0; q < kMaxDots; ++q) sum[q] = cmp[q] = 0.f;
  const long long len4 = len >> 2;
  const float4* wh = reinterpret_cast<const float4*>(w);
  const float4* wl = reinterpret_cast<const float4*>(w + len);
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < len4;
       e += (long long)gridDim.x * blockDim.x) {
    const float4 bh = wh[e], bl = wl[e];
#pragma unroll
    for (int q = 0; q < kMaxDots; ++q)
      if (q < nv) {
        const float4 ah = reinterpret_cast<const float4*>(V + q * stride)[e];
        const float4 al = reinterpret_cast<const float4*>(V + q * stride + len)[e];
        dot2_step(sum[q], cmp[q], ah.x, al.x, bh.x, bl.x);
        dot2_step(sum[q], cmp[q], ah.y, al.y, bh.y, bl.y);
        dot2_step(sum[q], cmp[q], ah.z, al.z, bh.z, bl.z);
        dot2_step(sum[q], cmp[q], ah.w, al.w, bh.w, bl.w);
      }
  }
  for (int q = 0; q < nv; ++q) {
    const FF r = block_sum_ff(ff_fast_two_sum(sum[q], cmp[q]), sh);
    if (threadIdx.x == 0) part[(long long)blockIdx.x * kMaxDots + q] = ff_to_double(r);
  }
}

// FP32 dot products of the high parts (the first Gram-Schmidt pass: the second, in
// float-float, removes what this one leaves)
__global__ void k_multidot_hi(const float* __restrict__ V, long long stride, int nv,
                              const float* __restrict__ w, long long len,
                              double* __restrict__ part) {
  __shared__ float sh[32];
  float acc[kMaxDots];
#pragma unroll
  for (int q = 0; q < kMaxDots; ++q) acc[q] = 0.f;
  const long long len4 = len >> 2;
  const float4* w4 = reinterpret_cast<const float4*>(w);
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < len4;
       e += (long long)gridDim.x * blockDim.x) {
    const float4 b = w4[e];
#pragma unroll
    for (int q = 0; q < kMaxDots; ++q)
      if (q < nv) {
        const float4 a = reinterpret_cast<const float4*>(V + q * stride)[e];
        acc[q] = fmaf(a.x, b.x, acc[q]);
        acc[q] = fmaf(a.y, b.y, acc[q]);
        acc[q] = fmaf(a.z, b.z, acc[q]);
        acc[q] = fmaf(a.w, b.w, acc[q]);
      }
  }
  for (int q = 0; q < nv; ++q) {
    const float r = block_sum(acc[q], sh);
    if (threadIdx.x == 0) part[(long long)blockIdx.x * kMaxDots + q] = (double)r;
  }
}

// Squared norm of a float-float vector with per-thread power-of-two scaling (the squares
// of entries above ~1e19 would overflow FP32): each thread keeps its sum scaled by 2^-2e,
// e the largest exponent it has seen, and rescales exactly when a larger one appears.
// Four consecutive entries per step; thread sums go to FP64 and are added in the fixed
// block order.
IPM_D void norm2_step(FF& acc, int& emax, float& scale, float xh, float xl) {
  if (xh == 0.f) return;
  int ex;
  frexpf(xh, &ex);
  ex = ex < -100 ? -100 : ex;  // keeps 2^-ex finite for subnormal entries
  if (ex > emax) {
    if (emax > -200) {
      const int d = 2 * (emax - ex);
      acc = FF{ldexpf(acc.h, d), ldexpf(acc.l, d)};
    }
    emax = ex;
    scale = ldexpf(1.f, -ex);  // exact power of two in [2^-128, 2^100]
  }
  const FF xs{xh * scale, xl * scale};
  acc = ff_add(acc, ff_mul(xs, xs));
}

__global__ void k_norm2_ff(const float* __restrict__ w, long long len, double* __restrict__ part) {
  __shared__ double sh[32];
  int emax = -200;
  float scale = 1.f;
  FF acc{0.f, 0.f};
  const long long len4 = len >> 2;
  const float4* wh = reinterpret_cast<const float4*>(w);
  const float4* wl = reinterpret_cast<const float4*>(w + len);
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < len4;
       e += (long long)gridDim.x * blockDim.x) {
    const float4 h = wh[e], l = wl[e];
    norm2_step(acc, emax, scale, h.x, l.x);
    norm2_step(acc, emax, scale, h.y, l.y);
    norm2_step(acc, emax, scale, h.z, l.z);
    norm2_step(acc, emax, scale, h.w, l.w);
  }
  double t = emax > -200 ? ldexp(ff_to_double(acc), 2 * emax) : 0.0;
  t = block_sum(t, sh);
  if (threadIdx.x == 0) part[(long long)blockIdx.x * kMaxDots] = t;
}

// FP64 sums of the block partials (block order); also the float-float value of each sum
// and, for `rsqrt`, of 1 / sqrt(sum) (a squared norm)
__global__ void k_reduce_dots_ff(const double* __restrict__ part, int nblocks, int nv,
                                 double* __restrict__ out, float* __restrict__ out_ff, int rsqrt) {
  __shared__ double sh[32];
  const int q = blockIdx.x;
  double acc = 0.0;
  for (int r = threadIdx.x; r < nblocks; r += blockDim.x) acc += part[(long long)r * kMaxDots + q];
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0) {
    out[q] = acc;
    const FF v = ff_from_double(rsqrt ? 1.0 / sqrt(acc) : acc);
    out_ff[2 * q] = v.h;
    out_ff[2 * q + 1] = v.l;
  }
}

// w += sign * sum_q coef[q] V_q (coef as float-float pairs), four entries per step
__global__ void k_axpy_multi_ff(float* __restrict__ w, const float* __restrict__ V,
                                long long stride, int nv, const float* __restrict__ coef,
                                float sign, long long len) {
  const long long len4 = len >> 2;
  float4* wh = reinterpret_cast<float4*>(w);
  float4* wl = reinterpret_cast<float4*>(w + len);
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < len4;
       e += (long long)gridDim.x * blockDim.x) {
    FF acc[4] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
    for (int q = 0; q < nv; ++q) {
      const FF cq{coef[2 * q], coef[2 * q + 1]};
      const float4 ah = reinterpret_cast<const float4*>(V + q * stride)[e];
      const float4 al = reinterpret_cast<const float4*>(V + q * stride + len)[e];
      acc[0] = ff_add(acc[0], ff_mul(cq, FF{ah.x, al.x}));
      acc[1] = ff_add(acc[1], ff_mul(cq, FF{ah.y, al.y}));
      acc[2] = ff_add(acc[2], ff_mul(cq, FF{ah.z, al.z}));
      acc[3] = ff_add(acc[3], ff_mul(cq, FF{ah.w, al.w}));
    }
    float4 h = wh[e], l = wl[e];
    FF r;
    r = ff_add(FF{h.x, l.x}, FF{sign * acc[0].h, sign * acc[0].l}); h.x = r.h; l.x = r.l;
    r = ff_add(FF{h.y, l.y}, FF{sign * acc[1].h, sign * acc[1].l}); h.y = r.h; l.y = r.l;
    r = ff_add(FF{h.z, l.z}, FF{sign * acc[2].h, sign * acc[2].l}); h.z = r.h; l.z = r.l;
    r = ff_add(FF{h.w, l.w}, FF{sign * acc[3].h, sign * acc[3].l}); h.w = r.h; l.w = r.l;
    wh[e] = h;
    wl[e] = l;
  }
}

// v *= f (f a float-float pair on the device)
__global__ void k_scale_ff(float* __restrict__ v, const float* __restrict__ f, long long len) {
  const FF s{f[0], f[1]};
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < len;
       e += (long long)gridDim.x * blockDim.x) {
    const FF r = ff_mul(ff_at(v, len, e), s);
    v[e] = r.h;
    v[len + e] = r.l;
  }
}

// out = a * x (FP64 in, float-float out) and back (FP64 out)
__global__ void k_to_ff(float* __restrict__ out, const double* __restrict__ x, double a,
                        long long len) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < len;
       e += (long long)gridDim.x * blockDim.x) {
    const FF r = ff_from_double(a * x[e]);
    out[e] = r.h;
    out[len + e] = r.l;
  }
}
__global__ void k_from_ff(double* __restrict__ out, const float* __restrict__ v, long long len) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < len;
       e += (long long)gridDim.x * blockDim.x)
    out[e] = ff_to_double(ff_at(v, len, e));
}

}  // namespace

// 4 x kRedBlocks blocks (memory-level parallelism); `hi` selects the FP32 dots of the
// high parts
void launch_multidot_ff(const float* V, long long stride, int nv, const float* w, long long len,
                        double* part, double* out, float* out_ff, int hi, cudaStream_t s) {
  const int nb = 4 * kRedBlocks;
  for (int q0 = 0; q0 < nv; q0 += kMaxDots) {
    int m = nv - q0 < kMaxDots ? nv - q0 : kMaxDots;
    count_launches(1);
    if (hi) k_multidot_hi<<<nb, kRedThreads, 0, s>>>(V + q0 * stride, stride, m, w, len, part);
    else k_multidot_ff<<<nb, kRedThreads, 0, s>>>(V + q0 * stride, stride, m, w, len, part);
    count_launches(1);
    k_reduce_dots_ff<<<m, 256, 0, s>>>(part, nb, m, out + q0, out_ff + 2 * q0, 0);
  }
}
void launch_norm2_ff(const float* w, long long len, double* part, double* out, float* out_ff,
                     cudaStream_t s) {
  count_launches(1);
  k_norm2_ff<<<4 * kRedBlocks, kRedThreads, 0, s>>>(w, len, part);
  count_launches(1);
  k_reduce_dots_ff<<<1, 256, 0, s>>>(part, 4 * kRedBlocks, 1, out, out_ff, 1);
}
void launch_axpy_multi_ff(float* w, const float* V, long long stride, int nv, const float* coef,
                          double sign, long long len, cudaStream_t s) {
  count_launches(1);
  k_axpy_multi_ff<<<vec_blocks(len / 4), 256, 0, s>>>(w, V, stride, nv, coef, (float)sign, len);
}
void launch_scale_ff(float* v, const float* f, long long len, cudaStream_t s) {
  count_launches(1);
  k_scale_ff<<<vec_blocks(len), 256, 0, s>>>(v, f, len);
}
void launch_to_ff(float* out, const double* x, double a, long long len, cudaStream_t s) {
  count_launches(1);
  k_to_ff<<<vec_blocks(len), 256, 0, s>>>(out, x, a, len);
}
void launch_from_ff(double* out, const float* v, long long len, cudaStream_t s) {
  count_launches(1);
  k_from_ff<<<vec_blocks(len), 256, 0, s>>>(out, v, len);
}
