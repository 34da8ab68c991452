// Serving loop: many independent interior point solves on one GPU.
//
// Worker threads each own a CUDA stream, so solves of different requests overlap on the
// device. A request is admitted when its solver fits the device-memory budget: solvers
// are pooled per (grid, state equation) and reset for each new request, idle solvers are
// evicted when a new grid needs room. Requests that arrive while others run are picked
// up as workers and memory free up (first admissible request in arrival order).
// Built on the public C ABI of ipm.h only.
#include <cuda_runtime.h>

#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <tuple>
#include <vector>

#include "ipm.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  long long id = 0;
  ipm_request rq{};
  std::vector<double> yd;
  size_t need = 0;
  bool done = false;
  int status = IPM_OK;
  ipm_report rep{};
  std::vector<double> u;
  Clock::time_point t_submit, t_start, t_end;
};

using Key = std::tuple<int, int, int, long long>;  // dim, n, kind, eps bits

Key key_of(const ipm_request& r) {
  long long eb = 0;
  double e = r.pde.kind == IPM_CONVDIFF_SUPG ? r.pde.eps : r.pde.kind == IPM_HEAT ? r.pde.T : 0.0;
  std::memcpy(&eb, &e, sizeof(eb));
  return Key{r.grid.dim, r.grid.n[0], r.pde.kind, eb};
}

// Device bytes a solver for this request will hold (upper estimate, mirroring its
// allocations: nodal fields, Krylov basis, both multigrid hierarchies, stencils).
size_t estimate_bytes(const ipm_request& r) {
  const long long n = r.grid.n[0];
  const long long pitch = (n + 31) / 32 * 32;
  const bool plane = r.grid.dim == 2 && r.pde.kind != IPM_HEAT;  // heat: n time levels
  const long long F = plane ? pitch * n : pitch * n * n;
  const long long nodes = plane ? n * n : n * n * n;
  const long long restart = r.opt.restart > 0 ? r.opt.restart : 50;
  double mg = r.grid.dim == 2 ? 4.0 / 3.0 : 8.0 / 7.0;
  double fields = 21 + 3 * 4 + 4 + 2 + 3 + 2 + 4  // state, data, diagonals, Krylov, buffers
                  + 0.5 * 2 + 0.5 * 4               // FP32 diagonals and Chebyshev
                  + mg * (5 * 1.0 + 5 * 0.5)        // FP64 + FP32 multigrid levels
                  + (2 * restart + 1) * 4.0;        // FGMRES V and Z
  if (r.pde.kind == IPM_CONVDIFF_SUPG) fields += mg * 9 * 1.5;
  double bytes = fields * (double)F * 8.0 + nodes * 8.0 + (8 << 20);
  return (size_t)(bytes * 1.1);
}

}  // namespace

struct ipm_server {
  int device = 0;
  size_t budget = 0;
  size_t used = 0;
  bool stop = false;
  long long next_id = 1;
  long long completed = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Request*> queue;
  std::map<long long, Request*> reqs;
  std::map<Key, std::vector<ipm_solver*>> idle;
  std::map<ipm_solver*, size_t> owned;  // every solver with its bytes
  std::vector<std::thread> workers;

  // take one idle solver (any grid) out of the pool into `dead`; the caller holds the lock
  // and destroys `dead` after releasing it (ipm_destroy frees device memory, which can
  // synchronise the device, and must not block the other workers)
  bool evict_one(std::vector<ipm_solver*>& dead) {
    for (auto& kv : idle) {
      if (kv.second.empty()) continue;
      ipm_solver* s = kv.second.back();
      kv.second.pop_back();
      used -= owned[s];
      owned.erase(s);
      dead.push_back(s);
      return true;
    }
    return false;
  }

  // first admissible request: a pooled solver is free, or its memory fits the budget
  // (evicting idle solvers of other grids when that makes room); caller holds the lock.
  // The budget is soft for pooled solvers: a reused solver's Krylov basis can grow during
  // its solve, and the growth is accounted when the solve ends.
  Request* admit(ipm_solver** reuse, std::vector<ipm_solver*>& dead) {
    for (auto it = queue.begin(); it != queue.end(); ++it) {
      Request* r = *it;
      auto pit = idle.find(key_of(r->rq));
      if (pit != idle.end() && !pit->second.empty()) {
        *reuse = pit->second.back();
        pit->second.pop_back();
        queue.erase(it);
        return r;
      }
      while (used + r->need > budget && evict_one(dead)) {
      }
      if (used + r->need <= budget) {
        used += r->need;
        *reuse = nullptr;
        queue.erase(it);
        return r;
      }
    }
    return nullptr;
  }

  void work() {
    cudaSetDevice(device);
    cudaStream_t st = nullptr;
    cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    while (true) {
      Request* r = nullptr;
      ipm_solver* s = nullptr;
      std::vector<ipm_solver*> dead;
      {
        std::unique_lock<std::mutex> lk(mu);
        cv_work.wait(lk, [&] { return stop || (r = admit(&s, dead)) != nullptr || !dead.empty(); });
      }
      for (ipm_solver* d : dead) ipm_destroy(d);  // outside the lock, before any new solver
      if (!r) {
        if (!dead.empty()) continue;  // evictions made room for nothing yet: look again
        break;
      }
      r->t_start = Clock::now();
      int rc = IPM_OK;
      bool fresh = s == nullptr;
      if (fresh) {
        rc = ipm_create(&r->rq.grid, &r->rq.pde, r->rq.alpha, r->rq.beta, &r->rq.bounds, &s);
        if (rc == IPM_OK) {
          std::lock_guard<std::mutex> lk(mu);
          size_t actual = ipm_device_bytes(s);
          used = used - r->need + actual;  // replace the estimate by the real footprint
          owned[s] = actual;
        } else {
          std::lock_guard<std::mutex> lk(mu);
          used -= r->need;
        }
      } else {
        rc = ipm_reset(s, r->rq.alpha, r->rq.beta, &r->rq.bounds);
      }
      if (rc == IPM_OK) rc = ipm_set_stream(s, st);
      if (rc == IPM_OK) rc = ipm_set_data(s, r->yd.data(), nullptr, nullptr);
      if (rc == IPM_OK) {
        rc = ipm_solve(s, &r->rq.opt, &r->rep);
        if (rc == IPM_OK || rc == IPM_ENOTCONV) {
          r->u.resize(r->yd.size());
          int g = ipm_get_control(s, r->u.data(), r->u.size());
          if (g != IPM_OK) rc = g;
        }
      }
      r->t_end = Clock::now();
      {
        std::lock_guard<std::mutex> lk(mu);
        if (s) {
          size_t b = ipm_device_bytes(s);  // the Krylov basis may have grown
          if (owned.count(s)) {
            used = used - owned[s] + b;
            owned[s] = b;
          }
          ipm_set_stream(s, nullptr);
          idle[key_of(r->rq)].push_back(s);
        }
        r->status = rc;
        r->done = true;
        ++completed;
      }
      cv_done.notify_all();
      cv_work.notify_all();
    }
    cudaStreamDestroy(st);
  }
};

extern "C" {

int ipm_server_create(int workers, size_t budget, ipm_server** out) {
  if (!out || workers < 1 || workers > 64 || budget == 0) return IPM_EINVAL;
  ipm_server* sv = new ipm_server();
  cudaGetDevice(&sv->device);
  sv->budget = budget;
  for (int i = 0; i < workers; ++i) sv->workers.emplace_back([sv] { sv->work(); });
  *out = sv;
  return IPM_OK;
}

int ipm_server_submit(ipm_server* sv, const ipm_request* rq, long long* ticket) {
  if (!sv || !rq || !ticket || !rq->yd) return IPM_EINVAL;
  if ((rq->grid.dim != 2 && rq->grid.dim != 3) || rq->grid.n[0] < 3) return IPM_EINVAL;
  if (rq->bounds.ua_v || rq->bounds.ub_v || rq->bounds.ya_v || rq->bounds.yb_v) return IPM_EINVAL;
  Request* r = new Request();
  r->rq = *rq;
  long long n = rq->grid.n[0];
  const bool plane = rq->grid.dim == 2 && rq->pde.kind != IPM_HEAT;
  r->yd.assign(rq->yd, rq->yd + (plane ? n * n : n * n * n));
  r->rq.yd = nullptr;
  r->need = estimate_bytes(*rq);
  r->t_submit = Clock::now();
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    if (r->need > sv->budget) {
      delete r;
      return IPM_ENOMEM;
    }
    r->id = sv->next_id++;
    sv->reqs[r->id] = r;
    sv->queue.push_back(r);
    *ticket = r->id;
  }
  sv->cv_work.notify_one();
  return IPM_OK;
}

int ipm_server_wait(ipm_server* sv, long long ticket, ipm_report* rep, double* u, size_t len,
                    double* latency_s, double* queue_s) {
  if (!sv) return IPM_EINVAL;
  std::unique_lock<std::mutex> lk(sv->mu);
  auto it = sv->reqs.find(ticket);
  if (it == sv->reqs.end()) return IPM_EINVAL;
  Request* r = it->second;
  sv->cv_done.wait(lk, [&] { return r->done; });
  sv->reqs.erase(it);
  lk.unlock();
  int rc = r->status;
  if (rep) *rep = r->rep;
  // a control exists only for a solve that ran (converged or not); any other status is
  // returned unchanged, without touching u
  if (u && (rc == IPM_OK || rc == IPM_ENOTCONV)) {
    if (len != r->u.size()) rc = IPM_EINVAL;
    else std::memcpy(u, r->u.data(), len * sizeof(double));
  }
  if (latency_s) *latency_s = std::chrono::duration<double>(r->t_end - r->t_submit).count();
  if (queue_s) *queue_s = std::chrono::duration<double>(r->t_start - r->t_submit).count();
  delete r;
  return rc;
}

int ipm_server_stats(ipm_server* sv, size_t* bytes_in_use, int* solvers, long long* completed) {
  if (!sv) return IPM_EINVAL;
  std::lock_guard<std::mutex> lk(sv->mu);
  if (bytes_in_use) *bytes_in_use = sv->used;
  if (solvers) *solvers = (int)sv->owned.size();
  if (completed) *completed = sv->completed;
  return IPM_OK;
}

void ipm_server_destroy(ipm_server* sv) {
  if (!sv) return;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->stop = true;
  }
  sv->cv_work.notify_all();
  for (auto& t : sv->workers) t.join();
  for (auto& kv : sv->owned) ipm_destroy(kv.first);
  for (auto& kv : sv->reqs) delete kv.second;
  delete sv;
}

}  // extern "C"
