// Request engine: continuous batching of solve requests on one GPU.
//
// Requests queue in arrival order and are admitted when a slot is free and
// the device memory they need (solve_footprint) fits in the budget.  A
// request that fits may be admitted ahead of older ones that do not
// (backfilling), unless the oldest waiting request has waited longer than
// kMaxBypassSeconds, after which admission is strictly in order until it
// is admitted -- so a large request is never starved by a stream of small
// ones.  Every
// admitted request gets its own stream and device state and advances by the
// same resumable solver as bridge_solve, so the kernels of different
// requests overlap on the GPU and a result is bit-identical alone or in a
// mix (deterministic reductions, fixed launch shapes).  One host thread
// drives all admitted requests; it only ever polls events, never blocks on
// one request while others could progress.  Copies between the caller's
// (pageable) host buffers and the device run on a separate I/O thread, and
// request buffers come from the stream-ordered pool, so neither a large copy
// nor a release stalls the other requests.  Smaller requests get
// higher-priority streams, so a quick solve is not queued behind the kernels
// of a large one.
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
// Phase of an active request: its upload is pending on the I/O thread, it is
// solving (engine thread), or its result download is pending.
enum ReqPhase { PH_UPLOAD = 0, PH_SOLVE = 1, PH_DOWNLOAD = 2 };

struct bridge_request_s {
  bridge_lattice_s* L = nullptr;
  bridge_op op{};
  bridge_solver prm{};
  int nrhs = 0;
  size_t bytes = 0;
  size_t nvals = 0;  // doubles per field (nrhs * V * 24)
  std::vector<double> b_host;
  const double* b_ref = nullptr;  // borrowed b (bridge_submit_borrowed): the caller's buffer, not copied
  // set by the engine thread
  int state = RQ_QUEUED;
  std::atomic<int> phase{PH_UPLOAD};
  int status = BRIDGE_PENDING;
  std::vector<double> x_host;
  std::atomic<bool> cancel{false};
  std::atomic<bool> released{false};
  std::string error;
  std::vector<bridge_info> info;
  double t_submit = 0, t_admit = 0, t_done = 0;
  cudaStream_t st = nullptr;
  std::unique_ptr<DevBuf> b_dev, x_dev;
  std::unique_ptr<SolveState> solve;
};

namespace {

struct Engine {
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<bridge_request_s*> queue;
  std::vector<bridge_request_s*> active;
  size_t budget = 0, used = 0;
  int max_active = 64;
  static constexpr double kMaxBypassSeconds = 2.0;
  bool started = false;
  std::thread th, io;
  std::mutex io_mu;
  std::condition_variable io_cv;
  std::deque<bridge_request_s*> io_queue;  // requests whose upload or download is pending

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
    io = std::thread([this, device] { io_loop(device); });
    io.detach();
  }

  // I/O thread: host <-> device copies of pageable buffers (synchronous for
  // the calling thread, so they must not run on the engine thread).
  void io_loop(int device) {
    cudaSetDevice(device);
    for (;;) {
      bridge_request_s* r;
      {
        std::unique_lock<std::mutex> lk(io_mu);
        io_cv.wait(lk, [this] { return !io_queue.empty(); });
        r = io_queue.front();
        io_queue.pop_front();
      }
      const size_t n = r->nvals * sizeof(double);
      if (r->phase.load() == PH_UPLOAD) {
        const double* src = r->b_ref ? r->b_ref : r->b_host.data();
        cudaError_t e = cudaMemcpyAsync(r->b_dev->ptr, src, n, cudaMemcpyHostToDevice, r->st);
        if (e == cudaSuccess && r->b_ref) e = cudaStreamSynchronize(r->st);  // the caller may reuse b after this
        if (e != cudaSuccess) {
          cudaGetLastError();
          r->error = std::string("upload: ") + cudaGetErrorString(e);
          r->cancel = true;
        }
        std::vector<double>().swap(r->b_host);  // staged by the copy above: the host copy is no longer needed
        r->phase.store(PH_SOLVE);             // queued ahead of every kernel of the solve
      } else {
        r->x_host.resize(r->nvals);
        cudaError_t e = cudaMemcpyAsync(r->x_host.data(), r->x_dev->ptr, n, cudaMemcpyDeviceToHost, r->st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(r->st);
        std::lock_guard<std::mutex> lk(mu);
        int status = r->status;
        std::string err = r->error;
        if (e != cudaSuccess) {
          cudaGetLastError();
          status = BRIDGE_ECUDA;
          err = std::string("download: ") + cudaGetErrorString(e);
        }
        finish(r, status, err);
        if (r->released) delete r;
        cv_done.notify_all();
      }
    }
  }

  void to_io(bridge_request_s* r) {
    std::lock_guard<std::mutex> lk(io_mu);
    io_queue.push_back(r);
    io_cv.notify_one();
  }

  void finish(bridge_request_s* r, int status, const std::string& err) {
    // engine mutex held by caller; the request's stream has no work a caller
    // waits for any more: its buffers return to the pool in stream order
    if (r->st) {
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

  // Stream priority from the work of the request (sites x right-hand sides):
  // small solves overtake the kernels of large ones on the GPU.
  static int priority_for(const bridge_request_s* r) {
    int least = 0, greatest = 0;
    cudaDeviceGetStreamPriorityRange(&least, &greatest);
    const double work = (double)r->L->V * r->nrhs;
    if (work <= (double)(1 << 21)) return greatest;
    if (work <= (double)(1 << 24)) return (least + greatest) / 2;
    return least;
  }

  void admit(bridge_request_s* r) {
    // called without the engine mutex; only the engine thread touches r's GPU state
    try {
      BR_CUDA(cudaStreamCreateWithPriority(&r->st, cudaStreamNonBlocking, priority_for(r)));
      const size_t n = r->nvals * sizeof(double);
      r->b_dev.reset(new DevBuf(n, r->st, true));
      r->x_dev.reset(new DevBuf(n, r->st, true));
      BR_CUDA(cudaMemsetAsync(r->x_dev->ptr, 0, n, r->st));
      {
        std::lock_guard<std::mutex> lk(r->L->api_mu);
        r->solve.reset(new SolveState(r->L, r->op, r->prm, r->nrhs, r->st, reinterpret_cast<double*>(r->b_dev->ptr),
                                      reinterpret_cast<double*>(r->x_dev->ptr)));
      }
      r->t_admit = now_seconds();
      r->phase.store(PH_UPLOAD);
      to_io(r);
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
        const bool strict = !queue.empty() && now_seconds() - queue.front()->t_submit > kMaxBypassSeconds;
        for (auto it = queue.begin(); it != queue.end() && (int)active.size() < max_active;) {
          bridge_request_s* r = *it;
          if (used + r->bytes > budget) {
            if (strict) break;  // the oldest request goes first
            ++it;
            continue;
          }
          it = queue.erase(it);
          r->state = RQ_ACTIVE;
          used += r->bytes;
          active.push_back(r);
          starting.push_back(r);
          if (strict) break;
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
        if (r->state != RQ_ACTIVE || !r->solve || r->phase.load() != PH_SOLVE) continue;
        bool done = false, ok = false;
        int status = BRIDGE_OK;
        std::string err;
        if (r->cancel) {
          done = true;
          status = BRIDGE_EINVAL;
          err = r->error.empty() ? "cancelled" : r->error;
        } else {
          try {
            if (r->solve->advance()) {
              done = ok = true;
              status = r->solve->status();
              r->info = r->solve->info();
            }
          } catch (const Error& e) {
            done = true;
            status = e.code;
            err = e.msg;
          }
        }
        if (!done) continue;
        progressed = true;
        std::lock_guard<std::mutex> lk(mu);
        active.erase(std::find(active.begin(), active.end(), r));
        if (ok) {
          // the solution goes back on the I/O thread, which then finishes the request
          r->status = status;
          r->phase.store(PH_DOWNLOAD);
          to_io(r);
        } else {
          finish(r, status, err);
          if (r->released) delete r;
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
                  bool borrow, bridge_request_h* out) {
  Engine& E = engine();
  auto* r = new bridge_request_s();
  r->L = L;
  r->op = op;
  r->prm = s;
  r->nrhs = nrhs;
  r->nvals = (size_t)nrhs * L->V * 24;
  r->bytes = solve_footprint(L, s, nrhs);
  if (borrow)
    r->b_ref = b;
  else
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
  L->in_flight.fetch_add(1);  // held from submission until the request is done or withdrawn
  *out = r;
  E.cv_work.notify_all();
  return BRIDGE_OK;
}
}  // namespace bridge

static int collect(bridge_request_s* r, double* x_out, bridge_info* info) {
  if (x_out && r->x_host.size() == r->nvals) std::memcpy(x_out, r->x_host.data(), r->nvals * sizeof(double));
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
  std::unique_lock<std::mutex> lk(E.mu);
  // a borrowed b may still be read by the upload of an admitted request: let that finish first
  while (h->b_ref && h->state == RQ_ACTIVE && h->phase.load() == PH_UPLOAD) {
    lk.unlock();
    std::this_thread::sleep_for(std::chrono::microseconds(100));
    lk.lock();
  }
  if (h->state == RQ_QUEUED) {
    auto it = std::find(E.queue.begin(), E.queue.end(), h);
    if (it != E.queue.end()) E.queue.erase(it);
    h->L->in_flight.fetch_sub(1);
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
