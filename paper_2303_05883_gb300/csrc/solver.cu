// Mixed-precision even-odd BiCGStab (Sec. 3 of the paper: BiCGStab for the
// clover operator, a mixed-precision BiCGStab for propagators; Eq. 1 for
// the even-odd preconditioning).
//
// Outer loop (FP64, on the GPU):  r = b - D x;  stop when ||r|| <= tol ||b||;
//   otherwise solve D e = r approximately in the inner precision and set
//   x += e (defect correction / iterative refinement).
// Inner solve of D e = r through Eq. 1:
//   b^_e = T_ee^-1 (r_e - D_eo T_oo^-1 r_o),  D^(eo) e_e = b^_e by BiCGStab,
//   e_o  = T_oo^-1 (r_o - D_oe e_e).
// BiCGStab (van der Vorst 1992), per iteration seven kernels:
//   v = D^ p  (two fused hop passes, <rhat, v> fused -> alpha on the GPU)
//   s = r - alpha v
//   t = D^ s  (<t, s>, |t|^2 fused -> omega)
//   x += alpha p + omega s; r = s - omega t  (<rhat, r>, |r|^2 -> beta, stop)
//   p = r + beta (p - omega v)
// All scalars stay on the device; the host copies them back once per batch
// of iterations, one batch behind the GPU, so the GPU never waits for it.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>

#include <nvtx3/nvToolsExt.h>

#include "solver.h"

namespace bridge {

extern std::atomic<long> g_launches;

// Small pinned host buffers are recycled through a process-wide free list:
// cudaFreeHost, like cudaFree, may synchronize the device, which would stall
// every concurrently running solve whenever one finishes.
namespace {
std::mutex g_pinned_mu;
std::multimap<size_t, void*> g_pinned_free;
size_t pinned_class(size_t n) {
  size_t c = 256;
  while (c < n) c <<= 1;
  return c;
}
}  // namespace

PinnedBuf::PinnedBuf(size_t n) {
  bytes = pinned_class(n);
  {
    std::lock_guard<std::mutex> lk(g_pinned_mu);
    auto it = g_pinned_free.find(bytes);
    if (it != g_pinned_free.end()) {
      ptr = it->second;
      g_pinned_free.erase(it);
    }
  }
  if (!ptr && cudaMallocHost(&ptr, bytes) != cudaSuccess) {
    cudaGetLastError();
    ptr = nullptr;
    throw Error{BRIDGE_ENOMEM, "cudaMallocHost failed"};
  }
  std::memset(ptr, 0, bytes);
}
PinnedBuf::~PinnedBuf() {
  if (!ptr) return;
  std::lock_guard<std::mutex> lk(g_pinned_mu);
  g_pinned_free.emplace(bytes, ptr);
}

static int inner_prec(const bridge_solver& prm) { return prm.mixed ? prm.inner_prec : P_F64; }
// Iterations a BiCGStab pass may take under BRIDGE_METHOD_AUTO before its
// progress decides whether the following passes switch to CG on the normal
// equations.
static constexpr long kAutoPassCap = 1000;
static int x_prec(int P) { return (P == P_F16 || P == P_BF16) ? P_F32 : P; }

size_t solve_footprint(const bridge_lattice_s* L, const bridge_solver& prm, int nrhs) {
  const int P = inner_prec(prm), PX = x_prec(P);
  const long vh = L->vh;
  const double sP = (double)spinor_block_bytes(P, vh), sX = (double)spinor_block_bytes(PX, vh),
               s64 = (double)spinor_block_bytes(P_F64, vh);
  double b = nrhs * (6 * s64        // b64, x64, r64 (full)
                     + 2 * sP       // rin (full)
                     + 7 * sP       // bh, r, rhat, p, v, s, t (even)
                     + sX + sP      // xin, xinp
                     + 2 * sP);     // tmp, eo (odd)
  b += nrhs * 2.0 * 2 * s64;        // canonical b and x held by the engine
  b += (double)nrhs * ((vh + 63) / 64) * 4 * 8 + 65536;
  return (size_t)b;
}

SolveState::SolveState(bridge_lattice_s* L, const bridge_op& op, const bridge_solver& prm, int nrhs, cudaStream_t st,
                       const double* b_dev, double* x_dev)
    : L_(L), op_(op), prm_(prm), nrhs_(nrhs), st_(st), b_dev_(b_dev), x_dev_(x_dev) {
  t0_ = std::chrono::steady_clock::now();
  P_ = inner_prec(prm_);
  PX_ = x_prec(P_);
  clover_ = op_is_clover(op_);
  kcsw_ = op_kcsw(op_);
  if (prm_.check_every <= 0) prm_.check_every = 16;
  if (prm_.max_outer <= 0) prm_.max_outer = 50;
  if (prm_.max_iter <= 0) prm_.max_iter = 20000;
  if (prm_.inner_tol <= 0) prm_.inner_tol = prm_.mixed ? (P_ == P_F32 ? 1e-5 : 2e-3) : std::max(prm_.tol * 0.25, 1e-15);
  cgnr_ = prm_.method == BRIDGE_METHOD_CGNR;
  batch_iters_ = prm_.check_every;
  if (L_->stats.profiling) {
    // event-timed runs launch exactly the iterations that execute
    batch_iters_ = 1;
    inflight_ = 1;
  }
  const long vh = L_->vh;
  b64_ = make_field(P_F64, BRIDGE_FULL, nrhs, vh, st_, true);
  x64_ = make_field(P_F64, BRIDGE_FULL, nrhs, vh, st_, true);
  r64_ = make_field(P_F64, BRIDGE_FULL, nrhs, vh, st_, true);
  rin_ = make_field(P_, BRIDGE_FULL, nrhs, vh, st_, true);
  bh_ = make_field(P_, BRIDGE_EVEN, nrhs, vh, st_, true);
  r_ = make_field(P_, BRIDGE_EVEN, nrhs, vh, st_, true);
  rhat_ = make_field(P_, BRIDGE_EVEN, nrhs, vh, st_, true);
  p_ = make_field(P_, BRIDGE_EVEN, nrhs, vh, st_, true);
  v_ = make_field(P_, BRIDGE_EVEN, nrhs, vh, st_, true);
  s_ = make_field(P_, BRIDGE_EVEN, nrhs, vh, st_, true);
  t_ = make_field(P_, BRIDGE_EVEN, nrhs, vh, st_, true);
  xin_ = make_field(PX_, BRIDGE_EVEN, nrhs, vh, st_, true);
  if (PX_ != P_) xinp_ = make_field(P_, BRIDGE_EVEN, nrhs, vh, st_, true);
  tmp_ = make_field(P_, BRIDGE_ODD, nrhs, vh, st_, true);
  eo_ = make_field(P_, BRIDGE_ODD, nrhs, vh, st_, true);
  scal_.reset(new DevBuf(sizeof(BiCGScalars) * nrhs, st_, true));
  partials_.reset(new DevBuf((size_t)nrhs * ((vh + 63) / 64) * 4 * sizeof(double), st_, true));
  counter_.reset(new DevBuf(256, st_, true));
  result_.reset(new DevBuf(sizeof(double) * 4 * 4 * nrhs, st_, true));
  mask_.reset(new DevBuf(sizeof(int) * nrhs, st_, true));
  for (int i = 0; i < 2; ++i) h_sc_[i].reset(new PinnedBuf(sizeof(BiCGScalars) * nrhs));
  cgsc_.reset(new DevBuf(sizeof(CGScalars) * nrhs, st_, true));
  for (int i = 0; i < 2; ++i) h_cg_[i].reset(new PinnedBuf(sizeof(CGScalars) * nrhs));
  h_cginit_.reset(new PinnedBuf(sizeof(CGScalars) * nrhs));
  h_result_.reset(new PinnedBuf(sizeof(double) * 4 * 4 * nrhs));
  h_mask_.reset(new PinnedBuf(sizeof(int) * nrhs));
  h_init_.reset(new PinnedBuf(sizeof(BiCGScalars) * nrhs));
  BR_CUDA(cudaEventCreateWithFlags(&ev_[0], cudaEventDisableTiming));
  BR_CUDA(cudaEventCreateWithFlags(&ev_[1], cudaEventDisableTiming));
  BR_CUDA(cudaEventCreateWithFlags(&ev_misc_, cudaEventDisableTiming));
  BR_CUDA(cudaMemsetAsync(counter_->ptr, 0, 256, st_));
  b2_.assign(nrhs, 0.0);
  r2_.assign(nrhs, 0.0);
  active_.assign(nrhs, 1);
  failed_.assign(nrhs, 0);
  stall_.assign(nrhs, 0);
  info_.assign(nrhs, bridge_info{});

  // make the operator data for this precision before any graph capture
  gauge_ptr(L_, P_);
  gauge_ptr(L_, P_F64);
  if (clover_) {
    clov_ = clover_set(L_, kcsw_);
    clover_ptr(L_, *clov_, P_, true);
    clover_ptr(L_, *clov_, P_F64, false);
  }
  if (st_ != L_->stream) BR_CUDA(cudaStreamSynchronize(L_->stream));
}

SolveState::~SolveState() {
  for (auto& g : graphs_)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  for (auto& e : ev_)
    if (e) cudaEventDestroy(e);
  if (ev_misc_) cudaEventDestroy(ev_misc_);
}

RedArgs SolveState::red(int fin, int slot) {
  RedArgs r;
  r.partials = reinterpret_cast<double*>(partials_->ptr);
  r.counter = reinterpret_cast<unsigned*>(counter_->ptr);
  r.sc = reinterpret_cast<BiCGScalars*>(scal_->ptr);
  r.result = reinterpret_cast<double*>(result_->ptr) + (long)slot * 4 * nrhs_;
  r.fin = fin;
  r.check_done = (fin == FIN_STORE || fin == FIN_INIT) ? 0 : 1;
  return r;
}

int SolveState::status() const {
  int st = BRIDGE_OK;
  for (const auto& i : info_)
    if (i.status != BRIDGE_OK) st = (st == BRIDGE_OK || i.status == BRIDGE_EBREAKDOWN) ? i.status : st;
  return st;
}

void SolveState::enqueue_residual() {
  nvtxRangePushA("bridge: FP64 residual");
  // r = b - T x + kappa H x (one launch per output parity), |r|^2 per parity
  for (int q = 0; q < 2; ++q) {
    HopCall c;
    c.prec = P_F64;
    c.flags = F_AUX | F_SELF | (clover_ ? F_SELF_CLOV : 0);
    c.red = R_NORM;
    c.cls = K_RESID;
    c.out_parity = q;
    c.nrhs = nrhs_;
    c.beta = op_.kappa;
    c.s1 = -1.0;
    c.caux = 1.0;
    c.kcsw = kcsw_;
    c.clov = clov_.get();
    for (int k = 0; k < 4; ++k) c.bc[k] = op_.bc[k];
    c.out = r64_.ptr(q);
    c.out_rs = r64_.rs;
    c.in = x64_.ptr(1 - q);
    c.in_rs = x64_.rs;
    c.self = x64_.ptr(q);
    c.self_rs = x64_.rs;
    c.aux = b64_.ptr(q);
    c.aux_rs = b64_.rs;
    c.redargs = red(FIN_STORE, 2 + q);
    run_hop(L_, c, st_);
  }
  BR_CUDA(cudaMemcpyAsync(h_result_->ptr, result_->ptr, sizeof(double) * 4 * 4 * nrhs_, cudaMemcpyDeviceToHost, st_));
  BR_CUDA(cudaEventRecord(ev_misc_, st_));
  pending_ = ev_misc_;
  nvtxRangePop();
}

void SolveState::launch_blas(int op, int cls, double bytes_per_site, double flops_per_site, int fin, bool count_work) {
  BlasArgs a;
  std::memset(&a, 0, sizeof(a));
  a.vh = (uint32_t)L_->vh;
  a.nrhs = nrhs_;
  a.x = xin_.ptr(0);
  a.x_rs = xin_.rs;
  a.r = r_.ptr(0);
  a.r_rs = r_.rs;
  a.p = p_.ptr(0);
  a.p_rs = p_.rs;
  a.v = v_.ptr(0);
  a.v_rs = v_.rs;
  a.s = s_.ptr(0);
  a.s_rs = s_.rs;
  a.t = t_.ptr(0);
  a.t_rs = t_.rs;
  a.rhat = rhat_.ptr(0);
  a.rhat_rs = rhat_.rs;
  a.b = bh_.ptr(0);
  a.b_rs = bh_.rs;
  a.red = red(fin);
  const std::string key = "blas/" + std::to_string(op) + "/" + std::to_string(P_) + "/" + std::to_string(L_->vh) + "/" +
                          std::to_string(nrhs_);
  LaunchShape sh = shape_for(L_, key, L_->vh, nrhs_, [&](int block) {
    int n = 0;
    bridge::launch_blas(op, P_, PX_, a, block, st_, &n);
    return n;
  });
  a.nblk = sh.nblk;
  const double n = count_work ? (double)L_->vh * nrhs_ : 0.0;
  note_launch(L_, cls, n * bytes_per_site, n * flops_per_site, st_, true);
  BR_CHECK(bridge::launch_blas(op, P_, PX_, a, sh.block, st_), BRIDGE_EINVAL, "blas variant");
  note_launch(L_, cls, 0, 0, st_, false);
  BR_CUDA(cudaGetLastError());
}

// Inner tolerance of the next pass of right-hand side r.  When the reduction
// still needed, tol / (current true relative residual), lies within a factor
// of ten below to four above the inner tolerance, this pass can be the last
// one: aim at half the needed reduction (at most the inner tolerance, at
// least a tenth of it), so that a small remainder does not cost one more
// pass with its FP64 residual.  Otherwise the inner tolerance.
double SolveState::pass_target(int r) const {
  const double t = prm_.inner_tol;
  if (outer_ == 0 || !(b2_[r] > 0.0) || !(r2_[r] > 0.0)) return t;
  const double need = prm_.tol / std::sqrt(r2_[r] / b2_[r]);
  if (need < 0.1 * t || need > 4.0 * t) return t;
  return std::min(t, std::max(0.5 * need, 0.1 * t));
}

void SolveState::begin_inner() {
  nvtxRangePushA("bridge: even-odd prepare + inner start");
  // mask: right-hand sides still above tolerance
  int* hm = reinterpret_cast<int*>(h_mask_->ptr);
  for (int r = 0; r < nrhs_; ++r) hm[r] = active_[r];
  BR_CUDA(cudaMemcpyAsync(mask_->ptr, hm, sizeof(int) * nrhs_, cudaMemcpyHostToDevice, st_));
  const int* mask = reinterpret_cast<const int*>(mask_->ptr);
  convert_field(L_, r64_, rin_, 0, st_, mask);
  convert_field(L_, r64_, rin_, 1, st_, mask);
  // b^_e = T_ee^-1 (r_e + kappa H_eo T_oo^-1 r_o)
  HopCall c;
  c.prec = P_;
  c.nrhs = nrhs_;
  c.kcsw = kcsw_;
  c.clov = clov_.get();
  for (int k = 0; k < 4; ++k) c.bc[k] = op_.bc[k];
  c.cls = K_PREP;
  c.out_parity = 0;
  c.beta = op_.kappa;
  c.caux = 1.0;
  c.out = bh_.ptr(0);
  c.out_rs = bh_.rs;
  c.aux = rin_.ptr(0);
  c.aux_rs = rin_.rs;
  if (clover_) {
    clover_site(L_, P_, true, kcsw_, 1, rin_, 1, tmp_, 1, nrhs_, st_, clov_.get());
    c.flags = F_AUX | F_E_CLOV;
    c.in = tmp_.ptr(1);
    c.in_rs = tmp_.rs;
  } else {
    c.flags = F_AUX;
    c.in = rin_.ptr(1);
    c.in_rs = rin_.rs;
  }
  run_hop(L_, c, st_);
  if (cgnr_) {
    begin_cgnr();
    nvtxRangePop();
    return;
  }
  // stage the per-rhs tolerance and iteration budget, then x = 0, r = rhat = p = b^
  BiCGScalars* hi = reinterpret_cast<BiCGScalars*>(h_init_->ptr);
  long left = std::max<long>(1, (long)prm_.max_iter - inner_total_);
  // automatic method: a BiCGStab pass gets a bounded budget so that a
  // stagnating one hands over to CG on the normal equations in time
  if (prm_.method == BRIDGE_METHOD_AUTO && (op_.kind == BRIDGE_WILSON || op_.kind == BRIDGE_CLOVER))
    left = std::min<long>(left, kAutoPassCap);
  for (int r = 0; r < nrhs_; ++r) {
    std::memset(&hi[r], 0, sizeof(BiCGScalars));
    const double t = pass_target(r);
    hi[r].tol2 = t * t;
    hi[r].max_iter = (int)std::min<long>(left, 1L << 30);
  }
  BR_CUDA(cudaMemcpyAsync(scal_->ptr, hi, sizeof(BiCGScalars) * nrhs_, cudaMemcpyHostToDevice, st_));
  const double S = P_ == P_F64 ? 192 : P_ == P_F32 ? 96 : 52, SX = PX_ == P_F64 ? 192 : PX_ == P_F32 ? 96 : 52;
  launch_blas(B_INIT, K_BLAS_INIT, 4 * S + SX, 24, FIN_INIT);
  batches_launched_ = batches_checked_ = 0;
  for (int k = 0; k < inflight_; ++k) enqueue_batch();
  nvtxRangePop();
}

void SolveState::enqueue_iteration() {
  if (cgnr_) {
    enqueue_cg_iteration();
    return;
  }
  const double S = P_ == P_F64 ? 192 : P_ == P_F32 ? 96 : 52, SX = PX_ == P_F64 ? 192 : PX_ == P_F32 ? 96 : 52;
  HopCall c;
  c.prec = P_;
  c.nrhs = nrhs_;
  c.kcsw = kcsw_;
  c.clov = clov_.get();
  for (int k = 0; k < 4; ++k) c.bc[k] = op_.bc[k];
  // pass 1 of D^: tmp_o = T_oo^-1 (-kappa H_oe in_e)
  HopCall p1 = c;
  p1.flags = clover_ ? F_E_CLOV : 0;
  p1.cls = K_DHAT1;
  p1.out_parity = 1;
  p1.beta = -op_.kappa;
  p1.out = tmp_.ptr(1);
  p1.out_rs = tmp_.rs;
  p1.redargs = red(FIN_NONE);
  p1.redargs.partials = nullptr;  // no reduction, but skip finished right-hand sides
  p1.count_work = false;          // executed iterations are credited in finish_inner
  // pass 2 of D^: out_e = in_e + kappa T_ee^-1 H_eo tmp_o
  HopCall p2 = c;
  p2.count_work = false;
  p2.flags = F_SELF | (clover_ ? F_E_CLOV : 0);
  p2.cls = K_DHAT2;
  p2.out_parity = 0;
  p2.beta = op_.kappa;
  p2.s1 = 1.0;
  p2.in = tmp_.ptr(1);
  p2.in_rs = tmp_.rs;
  // v = D^ p, alpha = rho / <rhat, v>
  p1.in = p_.ptr(0);
  p1.in_rs = p_.rs;
  run_hop(L_, p1, st_);
  p2.red = R_DOT_A;
  p2.cls = K_DHAT2A;
  p2.self = p_.ptr(0);
  p2.self_rs = p_.rs;
  p2.avec = rhat_.ptr(0);
  p2.avec_rs = rhat_.rs;
  p2.out = v_.ptr(0);
  p2.out_rs = v_.rs;
  p2.redargs = red(FIN_ALPHA);
  run_hop(L_, p2, st_);
  // s = r - alpha v
  launch_blas(B_S, K_BLAS_S, 3 * S, 48, FIN_NONE, false);
  // t = D^ s, omega = <t, s> / <t, t>
  p1.in = s_.ptr(0);
  p1.in_rs = s_.rs;
  run_hop(L_, p1, st_);
  p2.red = R_TS;
  p2.cls = K_DHAT2W;
  p2.self = s_.ptr(0);
  p2.self_rs = s_.rs;
  p2.avec = nullptr;
  p2.out = t_.ptr(0);
  p2.out_rs = t_.rs;
  p2.redargs = red(FIN_OMEGA);
  run_hop(L_, p2, st_);
  // x += alpha p + omega s, r = s - omega t, beta, convergence
  launch_blas(B_XR, K_BLAS_XR, 5 * S + 2 * SX, 192, FIN_RHO, false);
  // p = r + beta (p - omega v)
  launch_blas(B_P, K_BLAS_P, 4 * S, 96, FIN_NONE, false);
}

// ---------------------------------------------------------------- CGNR
// CG (Hestenes-Stiefel) on D^dag D^ e_e = D^dag b^_e, the normal equations of
// the Eq. 1 Schur system.  Past the critical kappa the spectrum of D^ can
// surround the origin, where BiCGStab (and any short-recurrence method on D^
// itself) stagnates; D^dag D^ is Hermitian positive definite for any
// non-singular D^, so CG converges, at a rate set by the condition number.
// The adjoint follows from gamma5-hermiticity of the hopping term,
// (H_oe)^dag = gamma5 H_eo gamma5, and T = T^dag commuting with gamma5:
//   D^dag v = v - gamma5 D_eo T_oo^-1 D_oe gamma5 T_ee^-1 v,
// three launches: s = gamma5 T_ee^-1 v; tmp = T_oo^-1 (-kappa H_oe s);
// out = v + kappa gamma5 H_eo tmp.
RedArgs SolveState::cg_red(int fin, bool check_done) {
  RedArgs r = red(fin);
  r.sc = nullptr;
  r.cg = reinterpret_cast<CGScalars*>(cgsc_->ptr);
  r.check_done = check_done ? 1 : 0;
  return r;
}

void SolveState::cg_dhat_norm(const Field& in, const Field& out) {
  HopCall c;
  c.prec = P_;
  c.nrhs = nrhs_;
  c.kcsw = kcsw_;
  c.clov = clov_.get();
  for (int k = 0; k < 4; ++k) c.bc[k] = op_.bc[k];
  c.count_work = false;
  c.flags = clover_ ? F_E_CLOV : 0;
  c.cls = K_DHAT1;
  c.out_parity = 1;
  c.beta = -op_.kappa;
  c.in = in.ptr(0);
  c.in_rs = in.rs;
  c.out = tmp_.ptr(1);
  c.out_rs = tmp_.rs;
  c.redargs = cg_red(FIN_NONE, true);
  c.redargs.partials = nullptr;  // no reduction, but skip finished right-hand sides
  run_hop(L_, c, st_);
  c.flags = F_SELF | (clover_ ? F_E_CLOV : 0);
  c.red = R_NORM;
  c.cls = K_DHAT2A;
  c.out_parity = 0;
  c.beta = op_.kappa;
  c.s1 = 1.0;
  c.in = tmp_.ptr(1);
  c.in_rs = tmp_.rs;
  c.self = in.ptr(0);
  c.self_rs = in.rs;
  c.out = out.ptr(0);
  c.out_rs = out.rs;
  c.redargs = cg_red(FIN_CG_ALPHA, true);
  run_hop(L_, c, st_);
}

void SolveState::cg_dhat_dag(const Field& in, const Field& out, bool check_done) {
  CopyArgs a;
  std::memset(&a, 0, sizeof(a));
  a.vh = (uint32_t)L_->vh;
  a.nrhs = nrhs_;
  a.g = L_->g;
  a.V = L_->V;
  a.nblk = (int)((L_->vh + 255) / 256);
  a.src = in.ptr(0);
  a.src_rs = in.rs;
  a.dst = s_.ptr(0);
  a.dst_rs = s_.rs;
  a.red = cg_red(FIN_NONE, check_done);
  const char* cl = clover_ ? clover_ptr(L_, *clov_, P_, true) : nullptr;  // parity 0 block first
  note_launch(L_, K_CLOVER, 0, 0, st_, true);
  BR_CHECK(launch_g5_site(P_, a, cl, 256, st_), BRIDGE_EINVAL, "precision");
  note_launch(L_, K_CLOVER, 0, 0, st_, false);
  BR_CUDA(cudaGetLastError());
  HopCall c;
  c.prec = P_;
  c.nrhs = nrhs_;
  c.kcsw = kcsw_;
  c.clov = clov_.get();
  for (int k = 0; k < 4; ++k) c.bc[k] = op_.bc[k];
  c.count_work = false;
  c.flags = clover_ ? F_E_CLOV : 0;
  c.cls = K_DHAT1;
  c.out_parity = 1;
  c.beta = -op_.kappa;
  c.in = s_.ptr(0);
  c.in_rs = s_.rs;
  c.out = tmp_.ptr(1);
  c.out_rs = tmp_.rs;
  c.redargs = cg_red(FIN_NONE, check_done);
  c.redargs.partials = nullptr;
  run_hop(L_, c, st_);
  c.flags = F_SELF | F_G5;
  c.cls = K_DHAT2;
  c.out_parity = 0;
  c.beta = op_.kappa;
  c.s1 = 1.0;
  c.in = tmp_.ptr(1);
  c.in_rs = tmp_.rs;
  c.self = in.ptr(0);
  c.self_rs = in.rs;
  c.out = out.ptr(0);
  c.out_rs = out.rs;
  run_hop(L_, c, st_);
}

void SolveState::begin_cgnr() {
  // r = D^dag b^ (the CG scalars of the previous pass are stale: no skipping)
  cg_dhat_dag(bh_, r_, false);
  CGScalars* hi = reinterpret_cast<CGScalars*>(h_cginit_->ptr);
  const long left = std::max<long>(1, (long)prm_.max_iter - inner_total_);
  for (int r = 0; r < nrhs_; ++r) {
    std::memset(&hi[r], 0, sizeof(CGScalars));
    hi[r].tol2 = prm_.inner_tol * prm_.inner_tol;
    hi[r].max_iter = (int)std::min<long>(left, 1L << 30);
  }
  BR_CUDA(cudaMemcpyAsync(cgsc_->ptr, hi, sizeof(CGScalars) * nrhs_, cudaMemcpyHostToDevice, st_));
  const double S = P_ == P_F64 ? 192 : P_ == P_F32 ? 96 : 52, SX = PX_ == P_F64 ? 192 : PX_ == P_F32 ? 96 : 52;
  {
    BlasArgs a;
    std::memset(&a, 0, sizeof(a));
    a.vh = (uint32_t)L_->vh;
    a.nrhs = nrhs_;
    a.x = xin_.ptr(0);
    a.x_rs = xin_.rs;
    a.r = r_.ptr(0);
    a.r_rs = r_.rs;
    a.p = p_.ptr(0);
    a.p_rs = p_.rs;
    a.red = cg_red(FIN_CG_INIT, false);
    const std::string key = "blas/" + std::to_string(B_CG_INIT) + "/" + std::to_string(P_) + "/" +
                            std::to_string(L_->vh) + "/" + std::to_string(nrhs_);
    LaunchShape sh = shape_for(L_, key, L_->vh, nrhs_, [&](int block) {
      int n = 0;
      bridge::launch_blas(B_CG_INIT, P_, PX_, a, block, st_, &n);
      return n;
    });
    a.nblk = sh.nblk;
    note_launch(L_, K_BLAS_INIT, (double)L_->vh * nrhs_ * (2 * S + SX), (double)L_->vh * nrhs_ * 24, st_, true);
    BR_CHECK(bridge::launch_blas(B_CG_INIT, P_, PX_, a, sh.block, st_), BRIDGE_EINVAL, "blas variant");
    note_launch(L_, K_BLAS_INIT, 0, 0, st_, false);
    BR_CUDA(cudaGetLastError());
  }
  batches_launched_ = batches_checked_ = 0;
  for (int k = 0; k < inflight_; ++k) enqueue_batch();
}

void SolveState::enqueue_cg_iteration() {
  // q = D^ p (v), alpha = |r|^2 / |q|^2
  cg_dhat_norm(p_, v_);
  // w = D^dag q (t)
  cg_dhat_dag(v_, t_, true);
  for (int op : {B_CG_XR, B_CG_P}) {
    BlasArgs a;
    std::memset(&a, 0, sizeof(a));
    a.vh = (uint32_t)L_->vh;
    a.nrhs = nrhs_;
    a.x = xin_.ptr(0);
    a.x_rs = xin_.rs;
    a.r = r_.ptr(0);
    a.r_rs = r_.rs;
    a.p = p_.ptr(0);
    a.p_rs = p_.rs;
    a.t = t_.ptr(0);
    a.t_rs = t_.rs;
    a.red = cg_red(op == B_CG_XR ? FIN_CG_BETA : FIN_NONE, true);
    const std::string key = "blas/" + std::to_string(op) + "/" + std::to_string(P_) + "/" + std::to_string(L_->vh) +
                            "/" + std::to_string(nrhs_);
    LaunchShape sh = shape_for(L_, key, L_->vh, nrhs_, [&](int block) {
      int n = 0;
      bridge::launch_blas(op, P_, PX_, a, block, st_, &n);
      return n;
    });
    a.nblk = sh.nblk;
    const int cls = op == B_CG_XR ? K_BLAS_XR : K_BLAS_P;
    note_launch(L_, cls, 0, 0, st_, true);
    BR_CHECK(bridge::launch_blas(op, P_, PX_, a, sh.block, st_), BRIDGE_EINVAL, "blas variant");
    note_launch(L_, cls, 0, 0, st_, false);
    BR_CUDA(cudaGetLastError());
  }
}

// Algorithmic work of the CG iterations that ran: per iteration two Schur
// first passes, the second pass with |q|^2, the adjoint's gamma5 T^-1 and
// second pass, and the two vector updates.
void SolveState::credit_cg_iterations(const std::vector<long>& iters) {
  long most = 0, sum = 0;
  for (long n : iters) {
    most = std::max(most, n);
    sum += n;
  }
  if (most == 0) return;
  const double vh = (double)L_->vh;
  const double S = P_ == P_F64 ? 192 : P_ == P_F32 ? 96 : 52, SX = PX_ == P_F64 ? 192 : PX_ == P_F32 ? 96 : 52;
  const double C = P_ == P_F64 ? 576 : P_ == P_F32 ? 288 : 144;
  const int f1 = clover_ ? F_E_CLOV : 0, f2 = F_SELF | (clover_ ? F_E_CLOV : 0);
  const HopCost h1 = hop_cost(P_, f1, R_NONE), hn = hop_cost(P_, f2, R_NORM), hd = hop_cost(P_, F_SELF, R_NONE);
  std::lock_guard<std::mutex> lk(L_->stats.mu);
  auto add = [&](int cls, double rhs_bytes, double shared_bytes, double rhs_flops) {
    L_->stats.k[cls].bytes += vh * (rhs_bytes * sum + shared_bytes * most);
    L_->stats.k[cls].flops += vh * rhs_flops * sum;
  };
  add(K_DHAT1, 2 * h1.rhs_bytes, 2 * h1.shared_bytes, 2 * h1.rhs_flops);
  add(K_DHAT2A, hn.rhs_bytes, hn.shared_bytes, hn.rhs_flops);
  add(K_DHAT2, hd.rhs_bytes, hd.shared_bytes, hd.rhs_flops);
  add(K_CLOVER, 2 * S, clover_ ? C : 0.0, clover_ ? 504 : 0);
  add(K_BLAS_XR, 4 * S + 2 * SX, 0, 96);
  add(K_BLAS_P, 3 * S, 0, 48);
}

void SolveState::capture_batch() {
  KStat before[K_NCLASS];
  {
    std::lock_guard<std::mutex> lk(L_->stats.mu);
    std::copy(std::begin(L_->stats.k), std::end(L_->stats.k), before);
  }
  const long l0 = g_launches.load();
  cudaGraph_t g = nullptr;
  BR_CUDA(cudaStreamBeginCapture(st_, cudaStreamCaptureModeThreadLocal));
  try {
    for (int it = 0; it < batch_iters_; ++it) enqueue_iteration();
  } catch (...) {
    cudaStreamEndCapture(st_, &g);
    if (g) cudaGraphDestroy(g);
    throw;
  }
  BR_CUDA(cudaStreamEndCapture(st_, &g));
  GraphRec& gr = graphs_[cgnr_ ? 1 : 0];
  cudaError_t e = cudaGraphInstantiate(&gr.exec, g, 0);
  cudaGraphDestroy(g);
  BR_CUDA(e);
  // nothing ran during capture: move the counted work into the per-replay delta
  std::lock_guard<std::mutex> lk(L_->stats.mu);
  for (int k = 0; k < K_NCLASS; ++k) {
    gr.delta[k].launches = L_->stats.k[k].launches - before[k].launches;
    gr.delta[k].bytes = L_->stats.k[k].bytes - before[k].bytes;
    gr.delta[k].flops = L_->stats.k[k].flops - before[k].flops;
    L_->stats.k[k] = before[k];
  }
  gr.launches = g_launches.load() - l0;
  g_launches.fetch_sub(gr.launches);
}

void SolveState::enqueue_batch() {
  nvtxRangePushA("bridge: BiCGStab batch");
  const bool use_graph = prm_.use_graph && !L_->stats.profiling;
  if (use_graph) {
    GraphRec& gr = graphs_[cgnr_ ? 1 : 0];
    if (!gr.exec) capture_batch();
    BR_CUDA(cudaGraphLaunch(gr.exec, st_));
    {
      std::lock_guard<std::mutex> lk(L_->stats.mu);
      for (int k = 0; k < K_NCLASS; ++k) {
        L_->stats.k[k].launches += gr.delta[k].launches;
        L_->stats.k[k].bytes += gr.delta[k].bytes;
        L_->stats.k[k].flops += gr.delta[k].flops;
      }
    }
    g_launches.fetch_add(gr.launches);
  } else {
    for (int it = 0; it < batch_iters_; ++it) enqueue_iteration();
  }
  const int slot = (int)(batches_launched_ & 1);
  if (cgnr_)
    BR_CUDA(cudaMemcpyAsync(h_cg_[slot]->ptr, cgsc_->ptr, sizeof(CGScalars) * nrhs_, cudaMemcpyDeviceToHost, st_));
  else
    BR_CUDA(cudaMemcpyAsync(h_sc_[slot]->ptr, scal_->ptr, sizeof(BiCGScalars) * nrhs_, cudaMemcpyDeviceToHost, st_));
  BR_CUDA(cudaEventRecord(ev_[slot], st_));
  ++batches_launched_;
  nvtxRangePop();
}

// Algorithmic work of the iterations that ran (launched iterations past
// convergence exit at once and move no data, so they are not counted).
void SolveState::credit_iterations(const std::vector<long>& iters) {
  long most = 0, sum = 0;
  for (long n : iters) {
    most = std::max(most, n);
    sum += n;
  }
  if (most == 0) return;
  const double vh = (double)L_->vh;
  const double S = P_ == P_F64 ? 192 : P_ == P_F32 ? 96 : 52, SX = PX_ == P_F64 ? 192 : PX_ == P_F32 ? 96 : 52;
  const int f1 = clover_ ? F_E_CLOV : 0, f2 = F_SELF | (clover_ ? F_E_CLOV : 0);
  const HopCost h1 = hop_cost(P_, f1, R_NONE), ha = hop_cost(P_, f2, R_DOT_A), ht = hop_cost(P_, f2, R_TS);
  std::lock_guard<std::mutex> lk(L_->stats.mu);
  auto add = [&](int cls, double rhs_bytes, double shared_bytes, double rhs_flops) {
    L_->stats.k[cls].bytes += vh * (rhs_bytes * sum + shared_bytes * most);
    L_->stats.k[cls].flops += vh * rhs_flops * sum;
  };
  add(K_DHAT1, 2 * h1.rhs_bytes, 2 * h1.shared_bytes, 2 * h1.rhs_flops);
  add(K_DHAT2A, ha.rhs_bytes, ha.shared_bytes, ha.rhs_flops);
  add(K_DHAT2W, ht.rhs_bytes, ht.shared_bytes, ht.rhs_flops);
  add(K_BLAS_S, 3 * S, 0, 48);
  add(K_BLAS_XR, 5 * S + 2 * SX, 0, 192);
  add(K_BLAS_P, 4 * S, 0, 96);
}

void SolveState::finish_inner() {
  nvtxRangePushA("bridge: reconstruct + accumulate");
  struct Pop {
    ~Pop() { nvtxRangePop(); }
  } pop;
  long most = 0;
  std::vector<long> iters(nrhs_, 0);
  bool stagnated = false;
  if (cgnr_) {
    const CGScalars* cg = reinterpret_cast<const CGScalars*>(h_cg_[(batches_checked_ - 1) & 1]->ptr);
    for (int r = 0; r < nrhs_; ++r) {
      if (!active_[r]) continue;
      info_[r].inner_iters += cg[r].iter;
      info_[r].cgnr_passes += 1;
      iters[r] = cg[r].iter;
      most = std::max<long>(most, cg[r].iter);
      if (cg[r].done == BREAKDOWN) info_[r].restarts += 1;
      stall_[r] = (cg[r].iter == 0) ? stall_[r] + 1 : 0;
    }
    inner_total_ += most;
    credit_cg_iterations(iters);
  } else {
    const BiCGScalars* sc = reinterpret_cast<const BiCGScalars*>(h_sc_[(batches_checked_ - 1) & 1]->ptr);
    for (int r = 0; r < nrhs_; ++r) {
      if (!active_[r]) continue;
      info_[r].inner_iters += sc[r].iter;
      iters[r] = sc[r].iter;
      most = std::max<long>(most, sc[r].iter);
      if (sc[r].done == BREAKDOWN) info_[r].restarts += 1;
      stall_[r] = (sc[r].iter == 0) ? stall_[r] + 1 : 0;
      // a pass that ended without reaching 1e-2 of its source: BiCGStab is
      // not converging on this spectrum
      if ((sc[r].done == MAXITER || sc[r].done == BREAKDOWN) && sc[r].r2 > 1e-4 * sc[r].b2) stagnated = true;
    }
    inner_total_ += most;
    credit_iterations(iters);
  }
  const int* mask = reinterpret_cast<const int*>(mask_->ptr);
  // e_o = T_oo^-1 (r_o + kappa H_oe e_e)
  const Field* xe = &xin_;
  if (PX_ != P_) {
    convert_field(L_, xin_, xinp_, 0, st_, mask);
    xe = &xinp_;
  }
  HopCall c;
  c.prec = P_;
  c.nrhs = nrhs_;
  c.kcsw = kcsw_;
  c.clov = clov_.get();
  for (int k = 0; k < 4; ++k) c.bc[k] = op_.bc[k];
  c.cls = K_PREP;
  c.flags = F_AUX | (clover_ ? F_E_CLOV : 0);
  c.out_parity = 1;
  c.beta = op_.kappa;
  c.caux = 1.0;
  c.in = xe->ptr(0);
  c.in_rs = xe->rs;
  c.aux = rin_.ptr(1);
  c.aux_rs = rin_.rs;
  c.out = eo_.ptr(1);
  c.out_rs = eo_.rs;
  run_hop(L_, c, st_);
  accumulate64(L_, xin_, 0, x64_, 0, st_, mask);
  accumulate64(L_, eo_, 1, x64_, 1, st_, mask);
  // the remaining passes run CG on the normal equations
  if (stagnated && prm_.method == BRIDGE_METHOD_AUTO) {
    cgnr_ = true;
    for (int r = 0; r < nrhs_; ++r) stall_[r] = 0;
  }
}

bool SolveState::advance() {
  for (;;) {
    if (pending_ != nullptr) {
      cudaError_t q = cudaEventQuery(pending_);
      if (q == cudaErrorNotReady) return false;
      BR_CUDA(q);
    }
    switch (state_) {
      case ST_START: {
        canon_to_field(L_, b_dev_, b64_, st_);
        canon_to_field(L_, x_dev_, x64_, st_);
        norm2_field(L_, b64_, 0, red(FIN_STORE, 0), st_);
        norm2_field(L_, b64_, 1, red(FIN_STORE, 1), st_);
        norm2_field(L_, x64_, 0, red(FIN_STORE, 2), st_);
        norm2_field(L_, x64_, 1, red(FIN_STORE, 3), st_);
        BR_CUDA(cudaMemcpyAsync(h_result_->ptr, result_->ptr, sizeof(double) * 4 * 4 * nrhs_, cudaMemcpyDeviceToHost, st_));
        BR_CUDA(cudaEventRecord(ev_misc_, st_));
        pending_ = ev_misc_;
        state_ = ST_BNORM;
        break;
      }
      case ST_BNORM: {
        double* hr = reinterpret_cast<double*>(h_result_->ptr);
        int* hm = reinterpret_cast<int*>(h_mask_->ptr);
        bool drop_guess = false, guess = false;
        for (int r = 0; r < nrhs_; ++r) {
          b2_[r] = hr[(0 * nrhs_ + r) * 4] + hr[(1 * nrhs_ + r) * 4];
          const double x2 = hr[(2 * nrhs_ + r) * 4] + hr[(3 * nrhs_ + r) * 4];
          hm[r] = b2_[r] > 0.0;  // the solution of D x = 0 is x = 0: drop the guess
          drop_guess = drop_guess || (b2_[r] == 0.0 && x2 != 0.0);
          guess = guess || (b2_[r] > 0.0 && x2 != 0.0);
        }
        if (drop_guess) {
          BR_CUDA(cudaMemcpyAsync(mask_->ptr, hm, sizeof(int) * nrhs_, cudaMemcpyHostToDevice, st_));
          canon_to_field(L_, x_dev_, x64_, st_, reinterpret_cast<const int*>(mask_->ptr));
        }
        if (guess) {
          enqueue_residual();
        } else {
          // x = 0 for every right-hand side: r = b exactly, no FP64 operator needed
          convert_field(L_, b64_, r64_, 0, st_, nullptr);
          convert_field(L_, b64_, r64_, 1, st_, nullptr);
          for (int r = 0; r < nrhs_; ++r) {
            hr[(2 * nrhs_ + r) * 4] = hr[(0 * nrhs_ + r) * 4];
            hr[(3 * nrhs_ + r) * 4] = hr[(1 * nrhs_ + r) * 4];
          }
          pending_ = nullptr;
        }
        state_ = ST_RESID;
        break;
      }
      case ST_RESID: {
        const double* hr = reinterpret_cast<const double*>(h_result_->ptr);
        bool any = false;
        for (int r = 0; r < nrhs_; ++r) {
          r2_[r] = hr[(2 * nrhs_ + r) * 4] + hr[(3 * nrhs_ + r) * 4];
          const double rel = b2_[r] > 0 ? std::sqrt(r2_[r] / b2_[r]) : std::sqrt(r2_[r]);
          info_[r].true_rel_residual = rel;
          info_[r].outer_iters = outer_;
          if (b2_[r] == 0.0 && r2_[r] == 0.0) active_[r] = 0;
          else if (!(rel > prm_.tol)) active_[r] = 0;
          else if (stall_[r] >= 2) {
            active_[r] = 0;
            failed_[r] = BRIDGE_EBREAKDOWN;
          }
          if (!std::isfinite(rel)) {
            active_[r] = 0;
            failed_[r] = BRIDGE_EBREAKDOWN;
          }
          any = any || active_[r];
        }
        if (!any || outer_ >= prm_.max_outer || inner_total_ >= prm_.max_iter) {
          for (int r = 0; r < nrhs_; ++r) {
            const double rel = info_[r].true_rel_residual;
            info_[r].status = failed_[r] ? failed_[r] : (rel <= prm_.tol || (b2_[r] == 0 && r2_[r] == 0)) ? BRIDGE_OK : BRIDGE_ENOCONV;
          }
          field_to_canon(L_, x64_, x_dev_, st_);
          BR_CUDA(cudaEventRecord(ev_misc_, st_));
          pending_ = ev_misc_;
          state_ = ST_FINISH;
          break;
        }
        ++outer_;
        begin_inner();
        pending_ = ev_[batches_checked_ & 1];
        state_ = ST_INNER;
        break;
      }
      case ST_INNER: {
        bool all = true;
        if (cgnr_) {
          const CGScalars* cg = reinterpret_cast<const CGScalars*>(h_cg_[batches_checked_ & 1]->ptr);
          for (int r = 0; r < nrhs_; ++r)
            if (cg[r].done == RUNNING) all = false;
        } else {
          const BiCGScalars* sc = reinterpret_cast<const BiCGScalars*>(h_sc_[batches_checked_ & 1]->ptr);
          for (int r = 0; r < nrhs_; ++r)
            if (sc[r].done == RUNNING) all = false;
        }
        ++batches_checked_;
        if (all) {
          finish_inner();
          enqueue_residual();
          state_ = ST_RESID;
        } else {
          enqueue_batch();
          pending_ = ev_[batches_checked_ & 1];
        }
        break;
      }
      case ST_FINISH: {
        const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0_).count();
        for (auto& i : info_) i.seconds = secs;
        pending_ = nullptr;
        state_ = ST_DONE;
        return true;
      }
      case ST_DONE:
        return true;
    }
  }
}

}  // namespace bridge
