// Krylov vector kernels over contiguous blocks of fields (FP64).
//
// Reductions run on a fixed grid (kRedBlocks x kRedThreads) with a fixed
// per-thread traversal order, so that every dot product is bitwise
// reproducible; partial sums are then added in block order.
#include "kernels.h"
#include <atomic>

static std::atomic<long long> g_launches{0};
void count_launches(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
long long launches_total() { return g_launches.load(std::memory_order_relaxed); }

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

__global__ void k_scale(double* __restrict__ y, const double* __restrict__ x,
                        const double* __restrict__ s, int invert, long long len) {
  double f = invert ? 1.0 / s[0] : s[0];
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < len;
       e += (long long)gridDim.x * blockDim.x)
    y[e] = x[e] * f;
}

__global__ void k_axpby(double* y, const double* x, double a, double b,
                        long long len) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < len;
       e += (long long)gridDim.x * blockDim.x)
    y[e] = b == 0.0 ? a * x[e] : a * x[e] + b * y[e];  // b = 0 never reads y
}

__global__ void k_axpy_dev(double* __restrict__ y, const double* __restrict__ x,
                           const double* __restrict__ a, double sign, long long len) {
  double f = sign * a[0];
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < len;
       e += (long long)gridDim.x * blockDim.x)
    y[e] += f * x[e];
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
void launch_scale(double* y, const double* x, const double* num, const double* den, int invert,
                  long long len, cudaStream_t s) {
  (void)num;
  count_launches(1);
  k_scale<<<vec_blocks(len), 256, 0, s>>>(y, x, den, invert, len);
}
void launch_axpby(double* y, const double* x, double a, double b, long long len, cudaStream_t s) {
  count_launches(1);
  k_axpby<<<vec_blocks(len), 256, 0, s>>>(y, x, a, b, len);
}
void launch_axpy_dev(double* y, const double* x, const double* a, double sign, long long len,
                     cudaStream_t s) {
  count_launches(1);
  k_axpy_dev<<<vec_blocks(len), 256, 0, s>>>(y, x, a, sign, len);
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
