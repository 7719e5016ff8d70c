// Even-odd preconditioned BiCGStab inside an FP64 defect-correction loop,
// written as a resumable state machine so that one code path serves both
// the blocking bridge_solve and the request engine (which interleaves many
// solves, each on its own stream).
#pragma once

#include <chrono>
#include <cmath>
#include <vector>

#include "host.h"

namespace bridge {

struct PinnedBuf {
  void* ptr = nullptr;
  size_t bytes = 0;
  explicit PinnedBuf(size_t n);
  ~PinnedBuf();
  PinnedBuf(const PinnedBuf&) = delete;
  PinnedBuf& operator=(const PinnedBuf&) = delete;
};

// Inner tolerance of the next defect-correction pass of a CG solve on the
// normal equations.  The first pass asks for `floor`; later passes ask only
// for the reduction still needed, tol |b| / |r|, corrected by the ratio
// `amp` between the reduction the true residual showed and the one the
// previous pass asked of the CG residual (the normal-equation residual
// under-reports the true one by up to the conditioning of the operator).
inline double next_inner_tol(double floor, double tol, double b2, double r2, double r2_prev, double tau_prev,
                             bool first) {
  if (first || !(r2 > 0.0) || !(r2_prev > 0.0) || !(tau_prev > 0.0)) return floor;
  double amp = std::sqrt(r2 / r2_prev) / tau_prev;
  amp = amp < 1.0 ? 1.0 : amp > 1e6 ? 1e6 : amp;
  const double want = tol * std::sqrt(b2 / r2);
  double tau = 0.5 * want / amp;
  if (tau > 0.1) tau = 0.1;
  return tau > floor ? tau : floor;
}

// Device bytes a solve of nrhs right-hand sides will hold (used for admission).
size_t solve_footprint(const bridge_lattice_s* L, const bridge_solver& prm, int nrhs);

class SolveState {
 public:
  // b_dev / x_dev: canonical FP64 full-lattice fields on the device (nrhs of
  // each).  x_dev holds the initial guess and receives the solution.
  SolveState(bridge_lattice_s* L, const bridge_op& op, const bridge_solver& prm, int nrhs, cudaStream_t st,
             const double* b_dev, double* x_dev);
  ~SolveState();

  // Queue whatever can be queued without blocking; true once finished.
  bool advance();
  // Event the caller may block on when advance() returned false.
  cudaEvent_t wait_event() const { return pending_; }
  const std::vector<bridge_info>& info() const { return info_; }
  int status() const;

 private:
  enum State { ST_START, ST_BNORM, ST_RESID, ST_INNER, ST_FINISH, ST_DONE };

  void enqueue_residual();
  void begin_inner();
  void enqueue_batch();
  void enqueue_iteration();
  void finish_inner();
  void launch_blas(int op, int cls, double bytes_per_site, double flops_per_site, int fin, bool count_work = true);
  void credit_iterations(const std::vector<long>& iters);
  void capture_batch();
  RedArgs red(int fin, int slot = 0);
  // CG on the normal equations of the Schur system (the inner method where
  // BiCGStab stagnates): D^ and its adjoint on even fields, the CG start
  // from the prepared source and one CG iteration.
  RedArgs cg_red(int fin, bool check_done);
  void cg_dhat_norm(const Field& in, const Field& out);
  void cg_dhat_dag(const Field& in, const Field& out, bool check_done);
  void begin_cgnr();
  void enqueue_cg_iteration();
  void credit_cg_iterations(const std::vector<long>& iters);

  bridge_lattice_s* L_;
  bridge_op op_;
  bridge_solver prm_;
  int nrhs_;
  cudaStream_t st_;
  const double* b_dev_;
  double* x_dev_;
  int P_, PX_;
  bool clover_;
  double kcsw_;
  std::shared_ptr<CloverSet> clov_;

  Field b64_, x64_, r64_, rin_, bh_, r_, rhat_, p_, v_, s_, t_, xin_, xinp_, tmp_, eo_;
  std::unique_ptr<DevBuf> scal_, partials_, counter_, result_, mask_;
  std::unique_ptr<PinnedBuf> h_sc_[2], h_result_, h_mask_, h_init_;
  cudaEvent_t ev_[2] = {nullptr, nullptr};
  cudaEvent_t ev_misc_ = nullptr;
  cudaEvent_t pending_ = nullptr;

  // one captured batch per inner method (0 BiCGStab, 1 CG on the normal equations)
  struct GraphRec {
    cudaGraphExec_t exec = nullptr;
    KStat delta[K_NCLASS];
    long launches = 0;
  } graphs_[2];
  bool cgnr_ = false;                      // the current inner pass runs CG on D^dag D^
  std::unique_ptr<DevBuf> cgsc_;           // CGScalars per right-hand side
  std::unique_ptr<PinnedBuf> h_cg_[2], h_cginit_;

  State state_ = ST_START;
  int outer_ = 0;
  long batches_launched_ = 0, batches_checked_ = 0;
  int batch_iters_ = 16;
  int inflight_ = 2;  // batches kept queued ahead of the host check
  long inner_total_ = 0;
  std::vector<double> b2_, r2_;
  double pass_target(int r) const;
  std::vector<int> active_, failed_, stall_;
  std::vector<bridge_info> info_;
  std::chrono::steady_clock::time_point t0_;
};

}  // namespace bridge
