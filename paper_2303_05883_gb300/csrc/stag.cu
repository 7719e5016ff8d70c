// Staggered operator and solver (host side and kernel instantiations).
//
// Even-odd blocks (Eq. 1 with D_ee = D_oo = m): D_eo, D_oe = the hopping
// term between parities, D^(eo) = 1 - D_eo D_oe / m^2.  The hopping term is
// anti-Hermitian, so m^2 - D_eo D_oe (the even-even block of D^dagger D) is
// Hermitian positive definite and the solve runs CG on it:
//   (m^2 - D_eo D_oe) x_e = m b_e - D_eo b_o,   x_o = (b_o - D_oe x_e) / m,
// in FP32 (or FP64) inside the FP64 defect correction r = b - D x, x += e.
// Per CG iteration four launches:
//   1 hop   t_o = D_oe p
//   2 hop   q = m^2 p - D_eo t_o,  Re <p, q> -> alpha = |r|^2 / <p, q>
//   3 vec   x += alpha p, r -= alpha q, |r|^2 -> beta
//   4 vec   p = r + beta p
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>

#include "solver.h"
#include "stag.cuh"
#include "stag.h"

namespace bridge {

bool op_is_staggered(const bridge_op& op) { return op.kind == BRIDGE_STAGGERED; }

void check_staggered(const bridge_op& op) {
  BR_CHECK(std::isfinite(op.mass) && op.mass != 0.0, BRIDGE_EINVAL, "op.mass must be finite and nonzero");
}

Field make_stag_field(int prec, int subset, int nrhs, long vh) {
  BR_CHECK(prec == P_F64 || prec == P_F32, BRIDGE_EINVAL, "staggered fields are F64 or F32");
  Field f;
  f.prec = prec;
  f.subset = subset;
  f.nrhs = nrhs;
  f.vh = vh;
  f.block = stag_block_bytes(prec, vh);
  f.rs = (subset == BRIDGE_FULL ? 2 : 1) * f.block;
  f.buf = std::make_shared<DevBuf>((size_t)(f.rs * (nrhs > 0 ? nrhs : 1)));
  return f;
}

Field& stag_workspace(bridge_lattice_s* L, const std::string& name, int prec, int subset, int nrhs) {
  const std::string key =
      "stag:" + name + "/" + std::to_string(prec) + "/" + std::to_string(subset) + "/" + std::to_string(nrhs);
  auto it = L->ws.find(key);
  if (it != L->ws.end()) return it->second;
  return L->ws.emplace(key, make_stag_field(prec, subset, nrhs, L->vh)).first->second;
}

// ------------------------------------------------------------ launches
namespace {

constexpr int kThreads = 256;

template <int P, int RED>
int hop_blocks_per_sm() {
  static int n = 0;
  if (n == 0) {
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, stag_hop_kernel<P, RED>, kThreads, 0);
    if (n <= 0) n = 1;
  }
  return n;
}

// Site blocks per right-hand side of a launch (persistent grid).
template <int P, int RED>
int hop_nblk(long vh, int nrhs) {
  const long cover = (vh + kThreads - 1) / kThreads;
  const long persist = (long)sm_count() * hop_blocks_per_sm<P, RED>() / std::max(1, nrhs);
  return (int)std::max<long>(1, std::min(cover, std::max<long>(persist, 1)));
}

int stag_nblk(int prec, int red, long vh, int nrhs) {
  if (prec == P_F64)
    return red == SR_NONE ? hop_nblk<P_F64, SR_NONE>(vh, nrhs)
           : red == SR_NORM ? hop_nblk<P_F64, SR_NORM>(vh, nrhs)
                            : hop_nblk<P_F64, SR_DOT_SELF>(vh, nrhs);
  return red == SR_NONE ? hop_nblk<P_F32, SR_NONE>(vh, nrhs)
         : red == SR_NORM ? hop_nblk<P_F32, SR_NORM>(vh, nrhs)
                          : hop_nblk<P_F32, SR_DOT_SELF>(vh, nrhs);
}

void launch_stag_hop(int prec, int red, StagArgs a, cudaStream_t st) {
  a.nblk = stag_nblk(prec, red, a.g.vh, a.nrhs);
  const unsigned grid = (unsigned)(a.nblk * a.nrhs);
  if (prec == P_F64) {
    if (red == SR_NONE) stag_hop_kernel<P_F64, SR_NONE><<<grid, kThreads, 0, st>>>(a);
    else if (red == SR_NORM) stag_hop_kernel<P_F64, SR_NORM><<<grid, kThreads, 0, st>>>(a);
    else stag_hop_kernel<P_F64, SR_DOT_SELF><<<grid, kThreads, 0, st>>>(a);
  } else {
    if (red == SR_NONE) stag_hop_kernel<P_F32, SR_NONE><<<grid, kThreads, 0, st>>>(a);
    else if (red == SR_NORM) stag_hop_kernel<P_F32, SR_NORM><<<grid, kThreads, 0, st>>>(a);
    else stag_hop_kernel<P_F32, SR_DOT_SELF><<<grid, kThreads, 0, st>>>(a);
  }
}

int vec_nblk(long vh, int nrhs) {
  const long cover = (vh + kThreads - 1) / kThreads;
  return (int)std::max<long>(1, std::min<long>(cover, (long)sm_count() * 8 / std::max(1, nrhs)));
}

template <int P, int PB>
void vec_dispatch(int op, const StagVecArgs& a, cudaStream_t st) {
  const unsigned grid = (unsigned)(a.nblk * a.nrhs);
  switch (op) {
    case SV_CGUPD: stag_vec_kernel<P, PB, SV_CGUPD><<<grid, kThreads, 0, st>>>(a); break;
    case SV_CGP: stag_vec_kernel<P, PB, SV_CGP><<<grid, kThreads, 0, st>>>(a); break;
    case SV_NORM: stag_vec_kernel<P, PB, SV_NORM><<<grid, kThreads, 0, st>>>(a); break;
    case SV_CONVERT: stag_vec_kernel<P, PB, SV_CONVERT><<<grid, kThreads, 0, st>>>(a); break;
    case SV_ACCUM: stag_vec_kernel<P, PB, SV_ACCUM><<<grid, kThreads, 0, st>>>(a); break;
    case SV_FROM_CANON: stag_vec_kernel<P, PB, SV_FROM_CANON><<<grid, kThreads, 0, st>>>(a); break;
    default: stag_vec_kernel<P, PB, SV_TO_CANON><<<grid, kThreads, 0, st>>>(a); break;
  }
}

void launch_stag_vec(int op, int prec, int precb, const StagVecArgs& a, cudaStream_t st) {
  if (prec == P_F64 && precb == P_F32) vec_dispatch<P_F64, P_F32>(op, a, st);
  else if (prec == P_F64) vec_dispatch<P_F64, P_F64>(op, a, st);
  else vec_dispatch<P_F32, P_F64>(op, a, st);
}

// One hop launch with its bookkeeping.
struct StagHop {
  int prec = P_F32, cls = K_STAG_HOP, red = SR_NONE, out_parity = 0, nrhs = 1;
  double scale = 0.5, s1 = 0.0, caux = 0.0;
  const char *in = nullptr, *self = nullptr, *aux = nullptr;
  char* out = nullptr;
  long in_rs = 0, out_rs = 0, self_rs = 0, aux_rs = 0;
  RedArgs redargs{};
};

void run_stag_hop(bridge_lattice_s* L, const bridge_op& op, const StagHop& c, cudaStream_t st) {
  StagArgs a;
  std::memset(static_cast<void*>(&a), 0, sizeof(a));
  a.g = L->g;
  a.out_parity = c.out_parity;
  a.nrhs = c.nrhs;
  a.scale = c.scale;
  a.scalef = (float)c.scale;
  a.s1 = c.s1;
  a.s1f = (float)c.s1;
  a.caux = c.caux;
  a.cauxf = (float)c.caux;
  for (int k = 0; k < 4; ++k) {
    a.bc[k] = op.bc[k];
    a.bcf[k] = (float)op.bc[k];
  }
  a.in = c.in;
  a.in_rs = c.in_rs;
  a.out = c.out;
  a.out_rs = c.out_rs;
  a.self = c.self;
  a.self_rs = c.self_rs;
  a.aux = c.aux;
  a.aux_rs = c.aux_rs;
  a.gauge = gauge_ptr(L, c.prec);
  a.red = c.redargs;
  if (c.red != SR_NONE && a.red.partials == nullptr) {
    ensure_red_scratch(L, (long)stag_nblk(c.prec, c.red, L->vh, c.nrhs) * c.nrhs, c.nrhs);
    a.red.partials = reinterpret_cast<double*>(L->red_partials->ptr);
    a.red.counter = reinterpret_cast<unsigned*>(L->red_counter->ptr);
    a.red.result = reinterpret_cast<double*>(L->red_result->ptr);
    if (a.red.fin == FIN_NONE) a.red.fin = FIN_STORE;
  }
  const double S = (double)stag_site_bytes(c.prec);
  const double per = S * (2 + (c.self ? 1 : 0) + (c.aux ? 1 : 0));
  const double links = 8.0 * (c.prec == P_F64 ? 144 : 48);
  const double bytes = (double)L->vh * (per * c.nrhs + links);
  const double flops = (double)L->vh * c.nrhs * (570 + (c.self ? 12 : 0) + (c.aux ? 12 : 0));
  note_launch(L, c.cls, bytes, flops, st, true);
  launch_stag_hop(c.prec, c.red, a, st);
  note_launch(L, c.cls, bytes, flops, st, false);
  BR_CUDA(cudaGetLastError());
}

StagVecArgs vec_args(bridge_lattice_s* L, int nrhs, int parity) {
  StagVecArgs a;
  std::memset(static_cast<void*>(&a), 0, sizeof(a));
  a.g = L->g;
  a.vh = (uint32_t)L->vh;
  a.nrhs = nrhs;
  a.nblk = vec_nblk(L->vh, nrhs);
  a.parity = parity;
  a.V = L->V;
  return a;
}

void run_vec(bridge_lattice_s* L, int op, int prec, int precb, StagVecArgs a, double bytes_per_site, cudaStream_t st) {
  const double bytes = (double)L->vh * a.nrhs * bytes_per_site;
  note_launch(L, K_STAG_VEC, bytes, 0, st, true);
  launch_stag_vec(op, prec, precb, a, st);
  note_launch(L, K_STAG_VEC, bytes, 0, st, false);
  BR_CUDA(cudaGetLastError());
}

}  // namespace

// ------------------------------------------------------------ conversions
void stag_canon_to_field(bridge_lattice_s* L, const double* canon, const Field& f, bool canon_full, cudaStream_t st) {
  const int lo = f.subset == BRIDGE_FULL ? 0 : f.subset, hi = f.subset == BRIDGE_FULL ? 1 : f.subset;
  for (int p = lo; p <= hi; ++p) {
    StagVecArgs a = vec_args(L, f.nrhs, p);
    a.canon = const_cast<double*>(canon);
    a.canon_full = canon_full;
    a.a = f.ptr(p);
    a.a_rs = f.rs;
    run_vec(L, SV_FROM_CANON, f.prec, P_F64, a, 48 + stag_site_bytes(f.prec), st);
  }
}

void stag_field_to_canon(bridge_lattice_s* L, const Field& f, double* canon, bool canon_full, cudaStream_t st) {
  const int lo = f.subset == BRIDGE_FULL ? 0 : f.subset, hi = f.subset == BRIDGE_FULL ? 1 : f.subset;
  for (int p = lo; p <= hi; ++p) {
    StagVecArgs a = vec_args(L, f.nrhs, p);
    a.canon = canon;
    a.canon_full = canon_full;
    a.a = f.ptr(p);
    a.a_rs = f.rs;
    run_vec(L, SV_TO_CANON, f.prec, P_F64, a, 48 + stag_site_bytes(f.prec), st);
  }
}

// ------------------------------------------------------------ operators
void stag_apply_deo(bridge_lattice_s* L, const bridge_op& op, int q, const Field& out, const Field& in,
                    cudaStream_t st) {
  StagHop h;
  h.prec = in.prec;
  h.out_parity = q;
  h.nrhs = in.nrhs;
  h.in = in.ptr(1 - q);
  h.in_rs = in.rs;
  h.out = out.ptr(q);
  h.out_rs = out.rs;
  run_stag_hop(L, op, h, st);
}

void stag_apply_d(bridge_lattice_s* L, const bridge_op& op, const Field& out, const Field& in, cudaStream_t st) {
  for (int q = 0; q < 2; ++q) {
    StagHop h;
    h.prec = in.prec;
    h.out_parity = q;
    h.nrhs = in.nrhs;
    h.in = in.ptr(1 - q);
    h.in_rs = in.rs;
    h.self = in.ptr(q);
    h.self_rs = in.rs;
    h.s1 = op.mass;
    h.out = out.ptr(q);
    h.out_rs = out.rs;
    run_stag_hop(L, op, h, st);
  }
}

void stag_apply_dhat(bridge_lattice_s* L, const bridge_op& op, const Field& out, const Field& in, cudaStream_t st) {
  Field& t = stag_workspace(L, "dhat_t", in.prec, BRIDGE_ODD, in.nrhs);
  StagHop h1;
  h1.prec = in.prec;
  h1.cls = K_STAG_PASS1;
  h1.out_parity = 1;
  h1.nrhs = in.nrhs;
  h1.in = in.ptr(0);
  h1.in_rs = in.rs;
  h1.out = t.ptr(1);
  h1.out_rs = t.rs;
  run_stag_hop(L, op, h1, st);
  StagHop h2;
  h2.prec = in.prec;
  h2.cls = K_STAG_PASS2;
  h2.out_parity = 0;
  h2.nrhs = in.nrhs;
  h2.scale = -0.5 / (op.mass * op.mass);
  h2.in = t.ptr(1);
  h2.in_rs = t.rs;
  h2.self = in.ptr(0);
  h2.self_rs = in.rs;
  h2.s1 = 1.0;
  h2.out = out.ptr(0);
  h2.out_rs = out.rs;
  run_stag_hop(L, op, h2, st);
}

// ------------------------------------------------------------ solver
int stag_solve(bridge_lattice_s* L, const bridge_op& op, const bridge_solver& prm, const double* b_dev, double* x_dev,
               int nrhs, bridge_info* info_out) {
  check_staggered(op);
  const auto t0 = std::chrono::steady_clock::now();
  cudaStream_t st = L->stream;
  const int P = prm.mixed ? prm.inner_prec : P_F64;
  BR_CHECK(P == P_F64 || P == P_F32, BRIDGE_EINVAL, "staggered solves run their inner CG in F64 or F32");
  const double m = op.mass, m2 = m * m;
  const double inner_tol = prm.inner_tol > 0 ? prm.inner_tol : (P == P_F64 ? std::max(prm.tol * 0.1, 1e-14) : 1e-6);
  const int max_outer = prm.max_outer > 0 ? prm.max_outer : 50;
  const int check_every = prm.check_every > 0 ? prm.check_every : 16;
  const long max_iter = prm.max_iter > 0 ? prm.max_iter : 20000;
  gauge_ptr(L, P_F64);
  gauge_ptr(L, P);

  Field b64 = make_stag_field(P_F64, BRIDGE_FULL, nrhs, L->vh), x64 = make_stag_field(P_F64, BRIDGE_FULL, nrhs, L->vh);
  Field r64 = make_stag_field(P_F64, BRIDGE_FULL, nrhs, L->vh);
  stag_canon_to_field(L, b_dev, b64, true, st);
  stag_canon_to_field(L, x_dev, x64, true, st);
  Field rin = make_stag_field(P, BRIDGE_FULL, nrhs, L->vh);
  Field bh = make_stag_field(P, BRIDGE_EVEN, nrhs, L->vh), cr = make_stag_field(P, BRIDGE_EVEN, nrhs, L->vh);
  Field xe = make_stag_field(P, BRIDGE_EVEN, nrhs, L->vh), pe = make_stag_field(P, BRIDGE_EVEN, nrhs, L->vh);
  Field qe = make_stag_field(P, BRIDGE_EVEN, nrhs, L->vh), to = make_stag_field(P, BRIDGE_ODD, nrhs, L->vh);
  Field eo = make_stag_field(P, BRIDGE_ODD, nrhs, L->vh);

  const long nblk_max = (L->vh + kThreads - 1) / kThreads;
  DevBuf sc(sizeof(CGScalars) * nrhs), partials(sizeof(double) * 4 * nblk_max * nrhs), counter(256);
  DevBuf mask(sizeof(int) * nrhs), resbuf(sizeof(double) * 4 * nrhs * 2);
  PinnedBuf h_sc(sizeof(CGScalars) * nrhs), h_res(sizeof(double) * 4 * nrhs * 2);
  BR_CUDA(cudaMemsetAsync(counter.ptr, 0, 256, st));
  auto red_of = [&](int fin, int check_done, double* result = nullptr) {
    RedArgs r;
    r.partials = reinterpret_cast<double*>(partials.ptr);
    r.counter = reinterpret_cast<unsigned*>(counter.ptr);
    r.cg = reinterpret_cast<CGScalars*>(sc.ptr);
    r.result = result;
    r.fin = fin;
    r.check_done = check_done;
    return r;
  };
  // |f|^2 per right-hand side of a full FP64 field
  auto norms = [&](const Field& f) {
    std::vector<double> out(nrhs, 0.0);
    for (int p = 0; p < 2; ++p) {
      StagVecArgs a = vec_args(L, nrhs, p);
      a.a = f.ptr(p);
      a.a_rs = f.rs;
      a.red = red_of(FIN_STORE, 0, reinterpret_cast<double*>(resbuf.ptr) + p * 4 * nrhs);
      run_vec(L, SV_NORM, P_F64, P_F64, a, 48, st);
    }
    BR_CUDA(cudaMemcpyAsync(h_res.ptr, resbuf.ptr, sizeof(double) * 8 * nrhs, cudaMemcpyDeviceToHost, st));
    BR_CUDA(cudaStreamSynchronize(st));
    const double* hr = static_cast<const double*>(h_res.ptr);
    for (int r = 0; r < nrhs; ++r) out[r] = hr[r * 4] + hr[4 * nrhs + r * 4];
    return out;
  };
  const std::vector<double> b2 = norms(b64);
  const std::vector<double> x02 = norms(x64);
  bool have_x = false;
  for (double v : x02) have_x = have_x || v != 0.0;

  std::vector<bridge_info> info(nrhs);
  for (auto& i : info) std::memset(&i, 0, sizeof(i));
  std::vector<int> done(nrhs, 0), failed(nrhs, 0), hmask(nrhs, 0);
  std::vector<double> r2(nrhs, 0.0), r2_prev(nrhs, 0.0), tau(nrhs, inner_tol);
  std::vector<int> passes(nrhs, 0);
  long total_iters = 0;
  for (int r = 0; r < nrhs; ++r)
    if (b2[r] == 0.0) {
      BR_CUDA(cudaMemsetAsync(x64.buf->ptr + (long)r * x64.rs, 0, x64.rs, st));
      done[r] = 1;
    }

  for (int outer = 0;; ++outer) {
    // ---- FP64 residual r = b - m x - H x
    const Field* defect = &b64;
    if (outer > 0 || have_x) {
      for (int q = 0; q < 2; ++q) {
        StagHop h;
        h.prec = P_F64;
        h.cls = K_STAG_RESID;
        h.red = SR_NORM;
        h.out_parity = q;
        h.nrhs = nrhs;
        h.scale = -0.5;
        h.in = x64.ptr(1 - q);
        h.in_rs = x64.rs;
        h.self = x64.ptr(q);
        h.self_rs = x64.rs;
        h.s1 = -m;
        h.aux = b64.ptr(q);
        h.aux_rs = b64.rs;
        h.caux = 1.0;
        h.out = r64.ptr(q);
        h.out_rs = r64.rs;
        h.redargs = red_of(FIN_STORE, 0, reinterpret_cast<double*>(resbuf.ptr) + q * 4 * nrhs);
        run_stag_hop(L, op, h, st);
      }
      BR_CUDA(cudaMemcpyAsync(h_res.ptr, resbuf.ptr, sizeof(double) * 8 * nrhs, cudaMemcpyDeviceToHost, st));
      BR_CUDA(cudaStreamSynchronize(st));
      const double* hr = static_cast<const double*>(h_res.ptr);
      for (int r = 0; r < nrhs; ++r) r2[r] = hr[r * 4] + hr[4 * nrhs + r * 4];
      defect = &r64;
    } else {
      r2 = b2;
    }
    bool any = false;
    for (int r = 0; r < nrhs; ++r) {
      if (b2[r] == 0.0) continue;
      const double rel = std::sqrt(r2[r] / b2[r]);
      info[r].true_rel_residual = rel;
      info[r].outer_iters = outer;
      if (!std::isfinite(rel)) failed[r] = 1;
      if (rel <= prm.tol) done[r] = 1;
      if (!done[r] && !failed[r]) any = true;
    }
    if (!any || outer >= max_outer || total_iters >= max_iter) break;

    // ---- inner solve of D e = defect for the active right-hand sides
    for (int r = 0; r < nrhs; ++r) hmask[r] = (!done[r] && !failed[r]) ? 1 : 0;
    BR_CUDA(cudaMemcpyAsync(mask.ptr, hmask.data(), sizeof(int) * nrhs, cudaMemcpyHostToDevice, st));
    for (int p = 0; p < 2; ++p) {
      StagVecArgs a = vec_args(L, nrhs, p);
      a.a = defect->ptr(p);
      a.a_rs = defect->rs;
      a.b = rin.ptr(p);
      a.b_rs = rin.rs;
      a.mask = reinterpret_cast<const int*>(mask.ptr);
      run_vec(L, SV_CONVERT, P_F64, P, a, 48 + stag_site_bytes(P), st);
    }
    // bh = m r_e - D_eo r_o
    {
      StagHop h;
      h.prec = P;
      h.cls = K_STAG_PREP;
      h.out_parity = 0;
      h.nrhs = nrhs;
      h.scale = -0.5;
      h.in = rin.ptr(1);
      h.in_rs = rin.rs;
      h.self = rin.ptr(0);
      h.self_rs = rin.rs;
      h.s1 = m;
      h.out = bh.ptr(0);
      h.out_rs = bh.rs;
      run_stag_hop(L, op, h, st);
    }
    {
      std::vector<CGScalars> hs(nrhs);
      for (int r = 0; r < nrhs; ++r) {
        CGScalars& g = hs[r];
        std::memset(&g, 0, sizeof(g));
        tau[r] = next_inner_tol(inner_tol, prm.tol, b2[r], r2[r], r2_prev[r], tau[r], passes[r] == 0);
        r2_prev[r] = r2[r];
        passes[r] += 1;
        g.tol2 = tau[r] * tau[r];
        g.max_iter = (int)std::max<long>(1, max_iter - total_iters);
      }
      BR_CUDA(cudaMemcpyAsync(sc.ptr, hs.data(), sizeof(CGScalars) * nrhs, cudaMemcpyHostToDevice, st));
    }
    // r = p = bh, x = 0, |bh|^2 -> FIN_CG_INIT
    BR_CUDA(cudaMemcpyAsync(cr.buf->ptr, bh.buf->ptr, cr.buf->bytes, cudaMemcpyDeviceToDevice, st));
    BR_CUDA(cudaMemcpyAsync(pe.buf->ptr, bh.buf->ptr, pe.buf->bytes, cudaMemcpyDeviceToDevice, st));
    BR_CUDA(cudaMemsetAsync(xe.buf->ptr, 0, xe.buf->bytes, st));
    {
      StagVecArgs a = vec_args(L, nrhs, 0);
      a.a = cr.ptr(0);
      a.a_rs = cr.rs;
      a.red = red_of(FIN_CG_INIT, 0);
      run_vec(L, SV_NORM, P, P_F64, a, stag_site_bytes(P), st);
    }
    auto iteration = [&]() {
      StagHop h1;
      h1.prec = P;
      h1.cls = K_STAG_PASS1;
      h1.out_parity = 1;
      h1.nrhs = nrhs;
      h1.in = pe.ptr(0);
      h1.in_rs = pe.rs;
      h1.out = to.ptr(1);
      h1.out_rs = to.rs;
      h1.redargs = red_of(FIN_NONE, 1);
      run_stag_hop(L, op, h1, st);
      StagHop h2;
      h2.prec = P;
      h2.cls = K_STAG_PASS2;
      h2.red = SR_DOT_SELF;
      h2.out_parity = 0;
      h2.nrhs = nrhs;
      h2.scale = -0.5;
      h2.in = to.ptr(1);
      h2.in_rs = to.rs;
      h2.self = pe.ptr(0);
      h2.self_rs = pe.rs;
      h2.s1 = m2;
      h2.out = qe.ptr(0);
      h2.out_rs = qe.rs;
      h2.redargs = red_of(FIN_CG_ALPHA, 1);
      run_stag_hop(L, op, h2, st);
      StagVecArgs u = vec_args(L, nrhs, 0);
      u.a = xe.ptr(0);
      u.b = cr.ptr(0);
      u.c = pe.ptr(0);
      u.d = qe.ptr(0);
      u.a_rs = u.b_rs = u.c_rs = u.d_rs = xe.rs;
      u.red = red_of(FIN_CG_BETA, 1);
      run_vec(L, SV_CGUPD, P, P_F64, u, 6 * stag_site_bytes(P), st);
      StagVecArgs v = vec_args(L, nrhs, 0);
      v.a = pe.ptr(0);
      v.b = cr.ptr(0);
      v.a_rs = v.b_rs = pe.rs;
      v.red = red_of(FIN_NONE, 1);
      run_vec(L, SV_CGP, P, P_F64, v, 3 * stag_site_bytes(P), st);
    };
    for (;;) {
      for (int k = 0; k < check_every; ++k) iteration();
      BR_CUDA(cudaMemcpyAsync(h_sc.ptr, sc.ptr, sizeof(CGScalars) * nrhs, cudaMemcpyDeviceToHost, st));
      BR_CUDA(cudaStreamSynchronize(st));
      const CGScalars* g = static_cast<const CGScalars*>(h_sc.ptr);
      bool running = false;
      for (int r = 0; r < nrhs; ++r) running = running || g[r].done == RUNNING;
      if (!running) break;
    }
    {
      const CGScalars* g = static_cast<const CGScalars*>(h_sc.ptr);
      long most = 0;
      for (int r = 0; r < nrhs; ++r) {
        if (!hmask[r]) continue;
        info[r].inner_iters += g[r].iter;
        most = std::max<long>(most, g[r].iter);
        if (g[r].done == BREAKDOWN) {
          info[r].restarts += 1;
          if (g[r].iter == 0) failed[r] = 1;
        }
      }
      total_iters += most;
    }
    // e_o = (r_o - D_oe x_e) / m, then x += e
    {
      StagHop h;
      h.prec = P;
      h.cls = K_STAG_PREP;
      h.out_parity = 1;
      h.nrhs = nrhs;
      h.scale = -0.5 / m;
      h.in = xe.ptr(0);
      h.in_rs = xe.rs;
      h.self = rin.ptr(1);
      h.self_rs = rin.rs;
      h.s1 = 1.0 / m;
      h.out = eo.ptr(1);
      h.out_rs = eo.rs;
      run_stag_hop(L, op, h, st);
    }
    for (int p = 0; p < 2; ++p) {
      const Field& src = p == 0 ? xe : eo;
      StagVecArgs a = vec_args(L, nrhs, p);
      a.a = src.ptr(p);
      a.a_rs = src.rs;
      a.b = x64.ptr(p);
      a.b_rs = x64.rs;
      a.mask = reinterpret_cast<const int*>(mask.ptr);
      run_vec(L, SV_ACCUM, P, P_F64, a, stag_site_bytes(P) + 96, st);
    }
  }

  stag_field_to_canon(L, x64, x_dev, true, st);
  BR_CUDA(cudaStreamSynchronize(st));
  const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  int status = BRIDGE_OK;
  for (int r = 0; r < nrhs; ++r) {
    info[r].seconds = secs;
    info[r].status = done[r] ? BRIDGE_OK : failed[r] ? BRIDGE_EBREAKDOWN : BRIDGE_ENOCONV;
    if (info[r].status != BRIDGE_OK)
      status = (status == BRIDGE_OK || info[r].status == BRIDGE_EBREAKDOWN) ? info[r].status : status;
    if (info_out) info_out[r] = info[r];
  }
  return status;
}

}  // namespace bridge
