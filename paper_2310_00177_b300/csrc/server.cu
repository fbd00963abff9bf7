// Continuous-batching solve server (npsolve_server_*, include/npsolve.h).
//
// Requests (a label grid and a right-hand side, any size divisible by
// 2^(L-1)) are queued as they arrive and admitted to solver slots as slots
// and memory become free.  Each slot owns a solver handle (its own workspace,
// Krylov state, image pyramid and kernel cache on the device), a non-blocking
// CUDA stream, device buffers for the request's labels / b / x, and a worker
// thread that runs the request's solve (npsolve_solve) on that stream.
// Solves of different slots therefore run concurrently on the GPU; a request
// that arrives while others are being solved starts as soon as a slot is free
// and its memory fits the HBM budget, without waiting for the others.
//
// Admission is first-fit in arrival order.  A slot's reservation is its
// measured device footprint (workspace + request buffers); before its first
// solve at a size it is the upper estimate kEstimateBytesPerCell bytes per
// cell.  A request is admitted only if the sum of all reservations, with the
// slot grown to the request's size, stays within the budget.  Results are
// deterministic: every slot runs the same kernels on the same sizes, so a
// request's x is identical whether it ran alone or among others.
#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/npsolve.h"
#include "nps_kernels.h"

namespace {

constexpr double kEstimateBytesPerCell = 256.0;  // upper bound of workspace + buffers per fine cell
constexpr size_t kEstimateFixedBytes = 64ull << 20;

using Clock = std::chrono::steady_clock;

struct Request {
  long long id = 0;
  int nx = 0, ny = 0, nz = 0;
  const uint8_t *lab = nullptr;  // caller's host buffers (valid until the result is read)
  const float *b = nullptr;
  double *x = nullptr;           // may be null: x is not copied back
  double tol = 1e-6;
  int max_iter = 1000;
  int iters = 0, status = -1;
  double relres = 0.0;
  Clock::time_point t_submit, t_start, t_end;
  long long cells() const { return (long long)nx * ny * nz; }
};

struct Slot {
  npsolve_t h = nullptr;
  cudaStream_t stream = nullptr;
  uint8_t *d_lab = nullptr;
  float *d_b = nullptr;
  double *d_x = nullptr;
  long long cap_cells = 0;   // capacity of the device request buffers
  long long ws_cells = 0;    // largest size the workspace has been grown to
  size_t reserved = 0;       // bytes counted against the budget
  Request *job = nullptr;
  bool busy = false;
  std::thread th;
};

size_t estimate_bytes(long long cells) { return (size_t)(kEstimateBytesPerCell * (double)cells) + kEstimateFixedBytes; }

}  // namespace

struct npsolve_server {
  npsolve_config cfg;
  std::vector<float> weights;
  size_t budget = 0;
  std::vector<Slot> slots;
  std::deque<Request *> queue;
  std::map<long long, Request *> reqs;
  std::vector<long long> finished;
  std::mutex mu;
  std::condition_variable cv;  // wakes workers (job assigned / stop)
  bool stop = false;
  long long next_id = 0;
  size_t reserved = 0, peak_reserved = 0;
  int device = 0;
  std::string err;
};

namespace {

int sfail(npsolve_server *s, int code, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (s) s->err = buf;
  nps::set_thread_error(buf);
  return code;
}

// Assign queued requests to free slots (first fit in arrival order) while
// the budget allows.  Called with s->mu held.
void dispatch_locked(npsolve_server *s) {
  for (auto it = s->queue.begin(); it != s->queue.end();) {
    Request *r = *it;
    int pick = -1;
    size_t pick_new = 0;
    for (int i = 0; i < (int)s->slots.size(); ++i) {
      Slot &sl = s->slots[i];
      if (sl.busy) continue;
      const size_t need = r->cells() <= sl.ws_cells ? sl.reserved : std::max(sl.reserved, estimate_bytes(r->cells()));
      if (s->reserved - sl.reserved + need > s->budget) continue;
      // prefer a slot that is already large enough (no growth)
      if (pick < 0 || (need == sl.reserved && pick_new != s->slots[pick].reserved)) {
        pick = i;
        pick_new = need;
      }
    }
    if (pick < 0) {
      ++it;
      continue;
    }
    Slot &sl = s->slots[pick];
    s->reserved = s->reserved - sl.reserved + pick_new;
    sl.reserved = pick_new;
    if (s->reserved > s->peak_reserved) s->peak_reserved = s->reserved;
    sl.job = r;
    sl.busy = true;
    it = s->queue.erase(it);
  }
  s->cv.notify_all();
}

void worker(npsolve_server *s, int idx) {
  Slot &sl = s->slots[idx];
  cudaSetDevice(s->device);
  for (;;) {
    Request *r = nullptr;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv.wait(lk, [&] { return s->stop || sl.job != nullptr; });
      if (s->stop && !sl.job) return;
      r = sl.job;
    }
    // The outputs go to locals first: a caller may call npsolve_server_result
    // as soon as r->status is non-negative, so r's fields are published (and
    // the status last) only under s->mu, below.
    const Clock::time_point t_start = Clock::now();
    const long long n = r->cells();
    int st = NPSOLVE_OK, iters = 0;
    double relres = 0.0;
    if (r->x) {
      // through the host-buffer call: the handle's staging buffers, b uploaded beside the setup
      st = npsolve_solve_host(sl.h, r->lab, r->nx, r->ny, r->nz, r->b, r->tol, r->max_iter, sl.stream, r->x,
                              &iters, &relres);
    } else if (n > sl.cap_cells) {  // grow this slot's request buffers
      cudaFree(sl.d_lab);
      cudaFree(sl.d_b);
      cudaFree(sl.d_x);
      sl.d_lab = nullptr;
      sl.d_b = nullptr;
      sl.d_x = nullptr;
      if (cudaMalloc(&sl.d_lab, n) != cudaSuccess || cudaMalloc(&sl.d_b, n * sizeof(float)) != cudaSuccess ||
          cudaMalloc(&sl.d_x, n * sizeof(double)) != cudaSuccess) {
        st = NPSOLVE_OOM;
        sl.cap_cells = 0;
      } else {
        sl.cap_cells = n;
      }
    }
    if (st == NPSOLVE_OK && !r->x) {
      cudaMemcpyAsync(sl.d_lab, r->lab, n, cudaMemcpyHostToDevice, sl.stream);
      cudaMemcpyAsync(sl.d_b, r->b, n * sizeof(float), cudaMemcpyHostToDevice, sl.stream);
      st = npsolve_solve(sl.h, sl.d_lab, r->nx, r->ny, r->nz, sl.d_b, r->tol, r->max_iter, sl.stream, sl.d_x,
                         &iters, &relres);
    }
    const Clock::time_point t_end = Clock::now();
    {
      std::lock_guard<std::mutex> lk(s->mu);
      r->iters = iters;
      r->relres = relres;
      r->t_start = t_start;
      r->t_end = t_end;
      r->status = st;
      if (n > sl.ws_cells) sl.ws_cells = n;
      // the measured footprint replaces the estimate
      const size_t actual = npsolve_workspace_bytes(sl.h) + (size_t)sl.cap_cells * (1 + sizeof(float) + sizeof(double));
      s->reserved = s->reserved - sl.reserved + actual;
      sl.reserved = actual;
      if (s->reserved > s->peak_reserved) s->peak_reserved = s->reserved;
      sl.job = nullptr;
      sl.busy = false;
      s->finished.push_back(r->id);
      dispatch_locked(s);
    }
  }
}

double ms_between(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double, std::milli>(b - a).count();
}

}  // namespace

extern "C" {

int npsolve_server_create(const npsolve_config *cfg, const float *weights_host, size_t n_weights,
                          size_t hbm_budget_bytes, int max_active, npsolve_server_t *out) {
  if (!cfg || !weights_host || !out || max_active < 1 || max_active > 64 || hbm_budget_bytes == 0)
    return sfail(nullptr, NPSOLVE_BAD_ARG, "bad argument");
  *out = nullptr;
  npsolve_server *s = new npsolve_server();
  s->cfg = *cfg;
  s->weights.assign(weights_host, weights_host + n_weights);
  s->budget = hbm_budget_bytes;
  cudaGetDevice(&s->device);
  s->slots.resize(max_active);
  for (int i = 0; i < max_active; ++i) {
    Slot &sl = s->slots[i];
    int st = npsolve_create(cfg, weights_host, n_weights, &sl.h);
    if (st != NPSOLVE_OK || cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess) {
      std::string msg = npsolve_last_error(nullptr);
      for (int j = 0; j <= i; ++j) {
        if (s->slots[j].h) npsolve_destroy(s->slots[j].h);
        if (s->slots[j].stream) cudaStreamDestroy(s->slots[j].stream);
      }
      delete s;
      return sfail(nullptr, st ? st : NPSOLVE_CUDA_ERROR, "server slot: %s", msg.c_str());
    }
  }
  for (int i = 0; i < max_active; ++i) s->slots[i].th = std::thread(worker, s, i);
  *out = s;
  return NPSOLVE_OK;
}

int npsolve_server_submit(npsolve_server_t s, const uint8_t *labels_host, int nx, int ny, int nz, const float *b_host,
                          double *x_host, double tol, int max_iter, long long *request_id) {
  if (!s || !labels_host || !b_host || !request_id) return sfail(s, NPSOLVE_BAD_ARG, "null argument");
  const int m = 1 << (s->cfg.levels - 1);
  if (nx < 1 || ny < 1 || nz < 1 || nx % m || ny % m || nz % m || (long long)nx * ny * nz > (1LL << 31) - 1)
    return sfail(s, NPSOLVE_BAD_DIMS, "dims %dx%dx%d not divisible by %d", nx, ny, nz, m);
  const long long n = (long long)nx * ny * nz;
  if (estimate_bytes(n) > s->budget) return sfail(s, NPSOLVE_OOM, "request larger than the HBM budget");
  Request *r = new Request();
  r->nx = nx;
  r->ny = ny;
  r->nz = nz;
  r->tol = tol;
  r->max_iter = max_iter;
  r->lab = labels_host;
  r->b = b_host;
  r->x = x_host;
  std::lock_guard<std::mutex> lk(s->mu);
  r->id = s->next_id++;
  r->t_submit = Clock::now();
  s->reqs[r->id] = r;
  s->queue.push_back(r);
  dispatch_locked(s);
  *request_id = r->id;
  return NPSOLVE_OK;
}

int npsolve_server_poll(npsolve_server_t s, long long *ids, int cap, int *count) {
  if (!s || !count || (cap > 0 && !ids)) return sfail(s, NPSOLVE_BAD_ARG, "null argument");
  std::lock_guard<std::mutex> lk(s->mu);
  const int m = (int)s->finished.size() < cap ? (int)s->finished.size() : cap;
  for (int i = 0; i < m; ++i) ids[i] = s->finished[i];
  s->finished.erase(s->finished.begin(), s->finished.begin() + m);
  *count = m;
  return NPSOLVE_OK;
}

int npsolve_server_result(npsolve_server_t s, long long id, int *iters, double *rel_residual, int *solve_status,
                          double *queue_ms, double *service_ms) {
  if (!s) return sfail(nullptr, NPSOLVE_BAD_ARG, "null server");
  Request *r = nullptr;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) return sfail(s, NPSOLVE_BAD_ARG, "unknown request %lld", id);
    r = it->second;
    if (r->status < 0) return sfail(s, NPSOLVE_BAD_ARG, "request %lld not finished", id);
    s->reqs.erase(it);
    // a result read before the poll that would have reported it: drop the id
    // from the finished list so that no later poll returns a released request
    for (auto f = s->finished.begin(); f != s->finished.end(); ++f)
      if (*f == id) {
        s->finished.erase(f);
        break;
      }
  }
  if (iters) *iters = r->iters;
  if (rel_residual) *rel_residual = r->relres;
  if (solve_status) *solve_status = r->status;
  if (queue_ms) *queue_ms = ms_between(r->t_submit, r->t_start);
  if (service_ms) *service_ms = ms_between(r->t_start, r->t_end);
  delete r;
  return NPSOLVE_OK;
}

int npsolve_server_stats(npsolve_server_t s, size_t *reserved_bytes, size_t *peak_reserved_bytes, int *active,
                         int *queued) {
  if (!s) return sfail(nullptr, NPSOLVE_BAD_ARG, "null server");
  std::lock_guard<std::mutex> lk(s->mu);
  if (reserved_bytes) *reserved_bytes = s->reserved;
  if (peak_reserved_bytes) *peak_reserved_bytes = s->peak_reserved;
  int a = 0;
  for (auto &sl : s->slots) a += sl.busy ? 1 : 0;
  if (active) *active = a;
  if (queued) *queued = (int)s->queue.size();
  return NPSOLVE_OK;
}

void npsolve_server_destroy(npsolve_server_t s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    s->queue.clear();
  }
  s->cv.notify_all();
  for (auto &sl : s->slots)
    if (sl.th.joinable()) sl.th.join();
  for (auto &sl : s->slots) {
    npsolve_destroy(sl.h);
    cudaStreamDestroy(sl.stream);
    cudaFree(sl.d_lab);
    cudaFree(sl.d_b);
    cudaFree(sl.d_x);
  }
  for (auto &kv : s->reqs) delete kv.second;
  delete s;
}

const char *npsolve_server_last_error(npsolve_server_t s) { return s ? s->err.c_str() : npsolve_last_error(nullptr); }

}  // extern "C"
