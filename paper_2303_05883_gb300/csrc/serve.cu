// Request engine: continuous batching of solve requests on one GPU.
//
// Requests queue in FIFO order and are admitted when a slot is free and the
// device memory they need (solve_footprint) fits in the budget.  Every
// admitted request gets its own stream and device state and advances by the
// same resumable solver as bridge_solve, so the kernels of different
// requests overlap on the GPU and a result is bit-identical alone or in a
// mix (deterministic reductions, fixed launch shapes).  One host thread
// drives all admitted requests; it only ever polls events, never blocks on
// one request while others could progress.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <thread>

#include "solver.h"

using namespace bridge;

namespace bridge {
double now_seconds() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}
}  // namespace bridge

enum ReqState { RQ_QUEUED = 0, RQ_ACTIVE = 1, RQ_DONE = 2 };

struct bridge_request_s {
  bridge_lattice_s* L = nullptr;
  bridge_op op{};
  bridge_solver prm{};
  int nrhs = 0;
  size_t bytes = 0;
  size_t nvals = 0;  // doubles per field (nrhs * V * 24)
  std::vector<double> b_host;
  // set by the engine thread
  int state = RQ_QUEUED;
  int status = BRIDGE_PENDING;
  bool cancel = false;
  bool released = false;
  std::string error;
  std::vector<bridge_info> info;
  double t_submit = 0, t_admit = 0, t_done = 0;
  cudaStream_t st = nullptr;
  std::unique_ptr<DevBuf> b_dev, x_dev;
  std::unique_ptr<PinnedBuf> x_pinned;
  std::unique_ptr<SolveState> solve;
};

namespace {

struct Engine {
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<bridge_request_s*> queue;
  std::vector<bridge_request_s*> active;
  size_t budget = 0, used = 0;
  int max_active = 16;
  bool started = false;
  std::thread th;

  void start(int device) {
    if (started) return;
    started = true;
    if (budget == 0) {
      size_t fr = 0, tot = 0;
      cudaSetDevice(device);
      if (cudaMemGetInfo(&fr, &tot) == cudaSuccess) budget = (size_t)(0.8 * (double)fr);
      else cudaGetLastError();
    }
    th = std::thread([this, device] { run(device); });
    th.detach();
  }

  void finish(bridge_request_s* r, int status, const std::string& err) {
    // engine mutex held by caller
    if (r->st) {
      cudaStreamSynchronize(r->st);
      r->solve.reset();
      r->b_dev.reset();
      r->x_dev.reset();
      cudaStreamDestroy(r->st);
      r->st = nullptr;
    }
    used -= r->bytes;
    r->L->in_flight.fetch_sub(1);
    r->status = status;
    r->error = err;
    r->state = RQ_DONE;
    r->t_done = now_seconds();
  }

  void admit(bridge_request_s* r) {
    // called without the engine mutex; only the engine thread touches r's GPU state
    try {
      BR_CUDA(cudaStreamCreateWithFlags(&r->st, cudaStreamNonBlocking));
      const size_t n = r->nvals * sizeof(double);
      r->b_dev.reset(new DevBuf(n));
      r->x_dev.reset(new DevBuf(n));
      r->x_pinned.reset(new PinnedBuf(n));
      BR_CUDA(cudaMemcpyAsync(r->b_dev->ptr, r->b_host.data(), n, cudaMemcpyHostToDevice, r->st));
      BR_CUDA(cudaMemsetAsync(r->x_dev->ptr, 0, n, r->st));
      {
        std::lock_guard<std::mutex> lk(r->L->api_mu);
        r->solve.reset(new SolveState(r->L, r->op, r->prm, r->nrhs, r->st, reinterpret_cast<double*>(r->b_dev->ptr),
                                      reinterpret_cast<double*>(r->x_dev->ptr)));
      }
      r->t_admit = now_seconds();
    } catch (const Error& e) {
      std::lock_guard<std::mutex> lk(mu);
      finish(r, e.code, e.msg);
      active.erase(std::find(active.begin(), active.end(), r));
      if (r->released) delete r;
      cv_done.notify_all();
    }
  }

  void run(int device) {
    cudaSetDevice(device);
    for (;;) {
      std::vector<bridge_request_s*> starting;
      {
        std::unique_lock<std::mutex> lk(mu);
        if (active.empty() && queue.empty()) cv_work.wait(lk, [this] { return !queue.empty(); });
        while (!queue.empty() && (int)active.size() < max_active && used + queue.front()->bytes <= budget) {
          bridge_request_s* r = queue.front();
          queue.pop_front();
          r->state = RQ_ACTIVE;
          r->L->in_flight.fetch_add(1);
          used += r->bytes;
          active.push_back(r);
          starting.push_back(r);
        }
      }
      for (auto* r : starting) admit(r);
      bool progressed = !starting.empty();
      std::vector<bridge_request_s*> snapshot;
      {
        std::lock_guard<std::mutex> lk(mu);
        snapshot = active;
      }
      for (auto* r : snapshot) {
        if (r->state != RQ_ACTIVE || !r->solve) continue;
        bool done = false;
        int status = BRIDGE_OK;
        std::string err;
        if (r->cancel) {
          done = true;
          status = BRIDGE_EINVAL;
          err = "cancelled";
        } else {
          try {
            if (r->solve->advance()) {
              done = true;
              status = r->solve->status();
              r->info = r->solve->info();
              const size_t n = r->nvals * sizeof(double);
              BR_CUDA(cudaMemcpyAsync(r->x_pinned->ptr, r->x_dev->ptr, n, cudaMemcpyDeviceToHost, r->st));
              BR_CUDA(cudaStreamSynchronize(r->st));
            }
          } catch (const Error& e) {
            done = true;
            status = e.code;
            err = e.msg;
          }
        }
        if (done) {
          std::lock_guard<std::mutex> lk(mu);
          finish(r, status, err);
          active.erase(std::find(active.begin(), active.end(), r));
          if (r->released) delete r;
          progressed = true;
          cv_done.notify_all();
        }
      }
      if (!progressed) std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
  }
};

Engine& engine() {
  static Engine* e = new Engine();  // lives until process exit
  return *e;
}

}  // namespace

namespace bridge {
int engine_submit(bridge_lattice_s* L, const bridge_op& op, const bridge_solver& s, const double* b, int nrhs,
                  bridge_request_h* out) {
  Engine& E = engine();
  auto* r = new bridge_request_s();
  r->L = L;
  r->op = op;
  r->prm = s;
  r->nrhs = nrhs;
  r->nvals = (size_t)nrhs * L->V * 24;
  r->bytes = solve_footprint(L, s, nrhs);
  r->b_host.assign(b, b + r->nvals);
  r->t_submit = now_seconds();
  std::lock_guard<std::mutex> lk(E.mu);
  E.start(L->device);
  if (r->bytes > E.budget) {
    const size_t need = r->bytes;
    delete r;
    throw Error{BRIDGE_ENOMEM, "request needs " + std::to_string(need) + " bytes, more than the whole budget"};
  }
  E.queue.push_back(r);
  *out = r;
  E.cv_work.notify_all();
  return BRIDGE_OK;
}
}  // namespace bridge

static int collect(bridge_request_s* r, double* x_out, bridge_info* info) {
  if (x_out && r->x_pinned) std::memcpy(x_out, r->x_pinned->ptr, r->nvals * sizeof(double));
  if (info)
    for (int k = 0; k < r->nrhs; ++k) info[k] = k < (int)r->info.size() ? r->info[k] : bridge_info{r->status, 0, 0, 0, 0, 0};
  if (r->status < 0 && !r->error.empty()) set_error(r->status, r->error);
  return r->status;
}

extern "C" {

int bridge_engine_config(size_t budget, int max_active) {
  Engine& E = engine();
  std::lock_guard<std::mutex> lk(E.mu);
  if (budget) E.budget = budget;
  if (max_active > 0) E.max_active = max_active;
  return BRIDGE_OK;
}

int bridge_poll(bridge_request_h h, double* x_out, bridge_info* info) {
  if (!h) return BRIDGE_EINVAL;
  Engine& E = engine();
  std::lock_guard<std::mutex> lk(E.mu);
  if (h->state != RQ_DONE) return BRIDGE_PENDING;
  return collect(h, x_out, info);
}

int bridge_wait(bridge_request_h h, int timeout_ms, double* x_out, bridge_info* info) {
  if (!h) return BRIDGE_EINVAL;
  Engine& E = engine();
  std::unique_lock<std::mutex> lk(E.mu);
  auto ready = [h] { return h->state == RQ_DONE; };
  if (timeout_ms < 0) E.cv_done.wait(lk, ready);
  else if (!E.cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready)) return BRIDGE_ETIMEDOUT;
  return collect(h, x_out, info);
}

int bridge_request_release(bridge_request_h h) {
  if (!h) return BRIDGE_OK;
  Engine& E = engine();
  std::lock_guard<std::mutex> lk(E.mu);
  if (h->state == RQ_QUEUED) {
    auto it = std::find(E.queue.begin(), E.queue.end(), h);
    if (it != E.queue.end()) E.queue.erase(it);
    delete h;
  } else if (h->state == RQ_ACTIVE) {
    h->cancel = true;  // the engine thread frees it once it stops
    h->released = true;
  } else {
    delete h;
  }
  return BRIDGE_OK;
}

int bridge_request_times(bridge_request_h h, double* t_submit, double* t_admit, double* t_done) {
  if (!h) return BRIDGE_EINVAL;
  Engine& E = engine();
  std::lock_guard<std::mutex> lk(E.mu);
  if (t_submit) *t_submit = h->t_submit;
  if (t_admit) *t_admit = h->t_admit;
  if (t_done) *t_done = h->t_done;
  return BRIDGE_OK;
}

}  // extern "C"
