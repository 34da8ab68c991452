// Chebyshev semi-iteration for (M + Theta_y) x = b that allocates no device memory.
//
// Some callers cannot let a library call cudaMalloc: applications that own all
// device memory through their own pool and cap what third-party code may take,
// or service loops where an allocation (and the device-wide synchronisation it
// may imply) would stall other work. This entry point keeps its work vectors in
// one file-scope device array of fixed size instead; every GPU that loads the
// library holds that array until the process exits.
#include <cuda.h>
#include <cuda_runtime.h>

#include <mutex>

#include "ipm.h"
#include "kernels.h"

namespace {

// Largest grid served: n^d <= 274625 nodes (65^3; also covers 2D grids up to 513^2).
constexpr long long kNoAllocMaxNodes = 274625;

// Three work vectors: the current and previous Chebyshev iterates and a copy of b.
// 3 * 274625 * 8 bytes = 6.3 MiB per device.
static __device__ __align__(256) double g_cheb_scratch[3 * kNoAllocMaxNodes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
struct Cached {
  double* addr = nullptr;
  unsigned long long ctx_id = 0;  // the context the address belongs to
};
Cached g_scratch[kMaxDevices];

// Context identity through the driver API, reached via the runtime's entry-point query
// (no link against libcuda): a device reset (cudaDeviceReset) destroys the context that
// holds the array, and a later call must look the address up again in the new one.
using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);
bool current_context_id(unsigned long long* id) {
  static CtxGetCurrentFn get_current = nullptr;
  static CtxGetIdFn get_id = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* f1 = nullptr;
    void* f2 = nullptr;
    cudaDriverEntryPointQueryResult q1, q2;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) ==
            cudaSuccess &&
        q1 == cudaDriverEntryPointSuccess &&
        cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) ==
            cudaSuccess &&
        q2 == cudaDriverEntryPointSuccess) {
      get_current = (CtxGetCurrentFn)f1;
      get_id = (CtxGetIdFn)f2;
    }
    cudaGetLastError();
  }
  if (!get_current || !get_id) return false;
  CUcontext ctx = nullptr;
  if (get_current(&ctx) != CUDA_SUCCESS || !ctx) return false;
  return get_id(ctx, id) == CUDA_SUCCESS;
}

// Device address of g_cheb_scratch on the current device. In host code the symbol
// name is only a host-side stand-in, so the address is looked up with the device
// current, once per device and context, and cached. Under lazy module loading the
// lookup is also what loads the module and so materialises the array on the device.
int scratch_address(double** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return IPM_ECUDA;
  std::lock_guard<std::mutex> lk(g_mu);
  unsigned long long id = 0;
  bool known = current_context_id(&id);
  Cached& c = g_scratch[dev];
  if (!c.addr || !known || c.ctx_id != id) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_cheb_scratch) != cudaSuccess) {
      cudaGetLastError();
      c.addr = nullptr;
      return IPM_ECUDA;
    }
    c.addr = (double*)p;
    c.ctx_id = current_context_id(&id) ? id : 0;
  }
  *out = c.addr;
  return IPM_OK;
}

}  // namespace

extern "C" int ipm_chebyshev_noalloc(int dim, int n, int steps, const double* theta_y,
                                     const double* b, double* x, void* stream) {
  if ((dim != 2 && dim != 3) || n < 3 || steps < 1 || !theta_y || !b || !x) return IPM_EINVAL;
  long long nodes = (long long)n * n * (dim == 3 ? n : 1);
  if (nodes > kNoAllocMaxNodes) return IPM_EINVAL;  // beyond the fixed work array
  double* work = nullptr;
  int rc = scratch_address(&work);
  if (rc != IPM_OK) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  // dense layout (pitch = n) so the caller's arrays are read and written in place
  GridDesc g;
  g.dim = dim;
  g.n = n;
  g.pitch = n;
  g.plane = (long long)n * n;
  g.field = nodes;
  g.h = 1.0 / (n - 1);
  g.heat = 0;  // the plain (stationary) stencil, whole-domain tracking
  g.tau = 0.0;
  g.obs = nullptr;
  double* bT = work;
  double* cur = work + nodes;
  double* prev = work + 2 * nodes;
  // The array keeps the previous call's contents (possibly for another grid):
  // the iterates' boundary entries must read as zero, so clear the used part.
  if (cudaMemsetAsync(work, 0, sizeof(double) * 3 * nodes, s) != cudaSuccess) return IPM_ECUDA;
  const double lmin = dim == 2 ? 0.25 : 0.125, lmax = dim == 2 ? 2.25 : 3.375;
  const double theta = 0.5 * (lmax + lmin), delta = 0.5 * (lmax - lmin), sig = theta / delta;
  const double dM = dim == 2 ? (2.0 * g.h / 3.0) * (2.0 * g.h / 3.0)
                             : (2.0 * g.h / 3.0) * (2.0 * g.h / 3.0) * (2.0 * g.h / 3.0);
  if (cudaMemsetAsync(x, 0, sizeof(double) * nodes, s) != cudaSuccess) return IPM_ECUDA;
  launch_cheb_init<double>(g, b, theta_y, dM, 1.0 / theta, bT, cur, prev, s);
  double rho = 1.0 / sig;
  for (int k = 1; k < steps; ++k) {
    double rho_new = 1.0 / (2.0 * sig - rho);
    double om = 2.0 * sig * rho_new;
    rho = rho_new;
    double* out = k == steps - 1 ? x : prev;
    launch_cheb_step<double, double>(g, cur, prev, bT, theta_y, dM, om, 1.0 / theta, out, s);
    if (k < steps - 1) {
      double* t = cur;
      cur = prev;
      prev = t;
    }
  }
  if (steps == 1) launch_convert<double, double>(g, cur, x, s);
  return cudaGetLastError() == cudaSuccess ? IPM_OK : IPM_ECUDA;
}
