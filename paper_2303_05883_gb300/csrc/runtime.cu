// Host runtime: device buffers, fields, gauge and clover storage, operator
// application, launch statistics and launch shapes.
#include <algorithm>
#include <cstring>
#include <string>

#include "host.h"

namespace bridge {

static thread_local std::string tl_last_error;
void set_error(int code, const std::string& msg) {
  (void)code;
  tl_last_error = msg;
}
const char* last_error_text() { return tl_last_error.c_str(); }

std::atomic<long> g_launches{0};
std::atomic<long> g_dev_allocs{0};

const char* kclass_name(int k) {
  static const char* names[K_NCLASS] = {"hop_deo",      "dirac_full",    "schur_pass1", "schur_pass2",
                                        "schur_pass2_alpha", "schur_pass2_omega", "evenodd_prep", "residual64",
                                        "blas_init",    "blas_s",        "blas_xr",     "blas_p",
                                        "convert",      "norm",          "clover_site", "setup",
                                        "dwf_mix",      "dwf_hop",       "dwf_schur_pass1", "dwf_schur_pass2",
                                        "dwf_schur_pass2_cg", "dwf_evenodd_prep", "dwf_residual64",
                                        "stag_hop",     "stag_pass1",    "stag_pass2",  "stag_vec",
                                        "stag_prep",    "stag_residual64",
                                        "mg_sap",       "mg_residual32", "mg_transfer", "mg_coarse",
                                        "mg_vec",       "mg_outer_dirac", "mg_setup"};
  return (k >= 0 && k < K_NCLASS) ? names[k] : "?";
}

// Keep freed stream-ordered memory in the pool (no release back to the
// driver between solves), once per device.
static void retain_pool_memory() {
  static std::mutex mu;
  static bool done[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(mu);
  if (dev < 0 || dev >= 64 || done[dev]) return;
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
    uint64_t thr = ~0ull;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
  }
  cudaGetLastError();
  done[dev] = true;
}

DevBuf::DevBuf(size_t n, cudaStream_t stream, bool stream_ordered) : st(stream), async(stream_ordered) {
  if (n == 0) return;
  cudaError_t e;
  if (async) {
    retain_pool_memory();
    e = cudaMallocAsync(reinterpret_cast<void**>(&ptr), n, st);
  } else {
    e = cudaMalloc(reinterpret_cast<void**>(&ptr), n);
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    ptr = nullptr;
    throw Error{BRIDGE_ENOMEM, "device allocation of " + std::to_string(n) + " bytes failed: " + cudaGetErrorString(e)};
  }
  bytes = n;
  g_dev_allocs.fetch_add(1);
}
DevBuf::~DevBuf() {
  if (!ptr) return;
  if (async)
    cudaFreeAsync(ptr, st);
  else
    cudaFree(ptr);
}

Field make_field(int prec, int subset, int nrhs, long vh, cudaStream_t st, bool stream_ordered) {
  Field f;
  f.prec = prec;
  f.subset = subset;
  f.nrhs = nrhs;
  f.vh = vh;
  f.block = spinor_block_bytes(prec, vh);
  f.rs = (subset == BRIDGE_FULL ? 2 : 1) * f.block;
  f.buf = std::make_shared<DevBuf>((size_t)(f.rs * (nrhs > 0 ? nrhs : 1)), st, stream_ordered);
  return f;
}

int sm_count() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 1;
  }
  return n;
}

// ----------------------------------------------------------- statistics
void note_launch(bridge_lattice_s* L, int cls, double bytes, double flops, cudaStream_t st, bool begin) {
  Stats& S = L->stats;
  std::lock_guard<std::mutex> lk(S.mu);
  if (begin) {
    g_launches.fetch_add(1);
    S.k[cls].launches += 1;
    S.k[cls].bytes += bytes;
    S.k[cls].flops += flops;
    if (S.profiling) {
      Stats::Rec r;
      r.cls = cls;
      if (S.pool.size() < 2) {
        cudaEvent_t e;
        for (int i = 0; i < 64; ++i) {
          cudaEventCreate(&e);
          S.pool.push_back(e);
        }
      }
      r.a = S.pool.back();
      S.pool.pop_back();
      r.b = S.pool.back();
      S.pool.pop_back();
      cudaEventRecord(r.a, st);
      S.recs.push_back(r);
    }
  } else if (S.profiling && !S.recs.empty()) {
    cudaEventRecord(S.recs.back().b, st);
  }
}

LaunchShape shape_for(bridge_lattice_s* L, const std::string& key, long vh, int nrhs,
                      const std::function<int(int)>& occ) {
  std::lock_guard<std::mutex> lk(L->tune_mu);
  LaunchShape s;
  auto it = L->tuned.find(key);
  if (it != L->tuned.end()) {
    s = it->second;
  } else {
    s.block = 128;
    const int per_sm = occ ? occ(s.block) : 0;
    const long resident = (long)sm_count() * (per_sm > 0 ? per_sm : 4);
    s.nblk = (int)std::max<long>(1, resident / std::max(1, nrhs));
    L->tuned[key] = s;
  }
  const long cover = (vh + s.block - 1) / s.block;
  if (s.nblk <= 0 || s.nblk > cover) s.nblk = (int)cover;
  return s;
}

void ensure_red_scratch(bridge_lattice_s* L, long n_partials, int nrhs) {
  size_t need = (size_t)n_partials * 4 * sizeof(double);
  if (!L->red_partials || L->red_partials->bytes < need) L->red_partials.reset(new DevBuf(need));
  size_t rneed = (size_t)(nrhs > 0 ? nrhs : 1) * 4 * sizeof(double);
  if (!L->red_result || L->red_result->bytes < rneed) L->red_result.reset(new DevBuf(rneed < 4096 ? 4096 : rneed));
  if (!L->red_counter) {
    L->red_counter.reset(new DevBuf(256));
    BR_CUDA(cudaMemsetAsync(L->red_counter->ptr, 0, 256, L->stream));
  }
}

// ------------------------------------------------------- gauge / clover
bool op_is_clover(const bridge_op& op) { return op.kind == BRIDGE_CLOVER && op.csw != 0.0 && op.kappa != 0.0; }
double op_kcsw(const bridge_op& op) { return op_is_clover(op) ? op.kappa * op.csw : 0.0; }

const char* gauge_ptr(bridge_lattice_s* L, int prec) {
  BR_CHECK(L->have_gauge, BRIDGE_ESTATE, "no gauge field uploaded");
  if (!L->gauge[prec]) {
    L->gauge[prec].reset(new DevBuf((size_t)(8 * link_block_bytes(prec, L->vh))));
    note_launch(L, K_SETUP, 0, 0, L->stream, true);
    BR_CHECK(launch_gauge_convert(prec, L->g, L->gauge[P_F64]->ptr, L->gauge[prec]->ptr, L->stream), BRIDGE_EINVAL,
             "gauge precision");
    note_launch(L, K_SETUP, 0, 0, L->stream, false);
    BR_CUDA(cudaGetLastError());
  }
  return L->gauge[prec]->ptr;
}

std::shared_ptr<CloverSet> clover_set(bridge_lattice_s* L, double kcsw) {
  BR_CHECK(L->have_gauge, BRIDGE_ESTATE, "no gauge field uploaded");
  std::lock_guard<std::mutex> lk(L->clover_mu);
  for (size_t i = 0; i < L->clovers.size(); ++i) {
    if (L->clovers[i]->kcsw == kcsw) {
      auto s = L->clovers[i];
      L->clovers.erase(L->clovers.begin() + i);
      L->clovers.insert(L->clovers.begin(), s);
      return s;
    }
  }
  auto s = std::make_shared<CloverSet>();
  s->kcsw = kcsw;
  const size_t n = (size_t)(2 * clover_block_bytes(P_F64, L->vh));
  s->T[P_F64].reset(new DevBuf(n));
  s->Tinv[P_F64].reset(new DevBuf(n));
  note_launch(L, K_SETUP, 0, 0, L->stream, true);
  launch_clover_build(L->g, L->gauge[P_F64]->ptr, kcsw, s->T[P_F64]->ptr, s->Tinv[P_F64]->ptr, L->stream);
  note_launch(L, K_SETUP, 0, 0, L->stream, false);
  BR_CUDA(cudaGetLastError());
  L->clovers.insert(L->clovers.begin(), s);
  const size_t keep = 4;  // sets still used by a solve stay alive through its reference
  if (L->clovers.size() > keep) L->clovers.resize(keep);
  return s;
}

const char* clover_ptr(bridge_lattice_s* L, CloverSet& set, int prec, bool inverse) {
  std::lock_guard<std::mutex> lk(set.mu);
  std::unique_ptr<DevBuf>* arr = inverse ? set.Tinv : set.T;
  if (!arr[prec]) {
    arr[prec].reset(new DevBuf((size_t)(2 * clover_block_bytes(prec, L->vh))));
    note_launch(L, K_SETUP, 0, 0, L->stream, true);
    BR_CHECK(launch_clover_convert(prec, L->g, arr[P_F64]->ptr, arr[prec]->ptr, L->stream), BRIDGE_EINVAL,
             "clover precision");
    note_launch(L, K_SETUP, 0, 0, L->stream, false);
    BR_CUDA(cudaGetLastError());
  }
  return arr[prec]->ptr;
}

const char* clover_ptr(bridge_lattice_s* L, int prec, bool inverse, double kcsw) {
  auto s = clover_set(L, kcsw);
  return clover_ptr(L, *s, prec, inverse);
}

// ------------------------------------------------------------ operators
static long spinor_site_bytes(int prec) { return prec == P_F64 ? 192 : prec == P_F32 ? 96 : 52; }
static long link_site_bytes(int prec) { return prec == P_F64 ? 144 : prec == P_F32 ? 48 : 24; }
static long clover_site_bytes(int prec) { return prec == P_F64 ? 576 : prec == P_F32 ? 288 : 144; }

HopCost hop_cost(int prec, int flags, int red) {
  const double S = (double)spinor_site_bytes(prec);
  double per_rhs = 2 * S;  // one input read, one output written
  if (flags & F_SELF) per_rhs += S;
  if (flags & F_AUX) per_rhs += S;
  if (red == R_DOT_A) per_rhs += S;
  double shared = 8.0 * link_site_bytes(prec);
  if (flags & F_E_CLOV) shared += clover_site_bytes(prec);
  if (flags & F_SELF_CLOV) shared += clover_site_bytes(prec);
  double fl = 1320 + 24;  // hop (8 projected hops) and the scale by beta
  if (flags & F_E_CLOV) fl += 504;
  if (flags & F_SELF_CLOV) fl += 504;
  if (flags & F_SELF) fl += 48;
  if (flags & F_AUX) fl += 48;
  if (red != R_NONE) fl += 48;
  return HopCost{per_rhs, shared, fl};
}

static std::string dims_key(const bridge_lattice_s* L) {
  return std::to_string(L->dims[0]) + "x" + std::to_string(L->dims[1]) + "x" + std::to_string(L->dims[2]) + "x" +
         std::to_string(L->dims[3]);
}

void run_hop(bridge_lattice_s* L, HopCall c, cudaStream_t st) {
  HopArgs a;
  std::memset(&a, 0, sizeof(a));
  a.g = L->g;
  a.out_parity = c.out_parity;
  a.nrhs = c.nrhs;
  a.beta = c.beta;
  a.s1 = c.s1;
  a.caux = c.caux;
  for (int k = 0; k < 4; ++k) a.bc[k] = (double)c.bc[k];
  a.out = c.out;
  a.out_rs = c.out_rs;
  a.in = c.in;
  a.in_rs = c.in_rs;
  a.self = c.self;
  a.self_rs = c.self_rs;
  a.aux = c.aux;
  a.aux_rs = c.aux_rs;
  a.avec = c.avec;
  a.avec_rs = c.avec_rs;
  a.gauge = gauge_ptr(L, c.prec);
  if (c.flags & (F_E_CLOV | F_SELF_CLOV)) {
    std::shared_ptr<CloverSet> keep;
    CloverSet* cs = c.clov;
    if (!cs) {
      keep = clover_set(L, c.kcsw);
      cs = keep.get();
    }
    a.clovE = (c.flags & F_E_CLOV) ? clover_ptr(L, *cs, c.prec, true) : nullptr;
    a.clovM = (c.flags & F_SELF_CLOV) ? clover_ptr(L, *cs, c.prec, false) : nullptr;
  }
  const std::string key = "hop/" + std::to_string(c.prec) + "/" + std::to_string(c.flags) + "/" +
                          std::to_string(c.red) + "/" + dims_key(L) + "/" + std::to_string(c.nrhs);
  LaunchShape sh = shape_for(L, key, L->vh, c.nrhs, [&](int block) {
    int n = 0;
    launch_hop_any(c.prec, c.flags, c.red, a, block, st, &n, 0);
    return n;
  });
  a.nblk = sh.nblk;
  a.red = c.redargs;
  if (c.red != R_NONE && a.red.partials == nullptr) {
    ensure_red_scratch(L, (long)sh.nblk * c.nrhs, c.nrhs);
    a.red.partials = reinterpret_cast<double*>(L->red_partials->ptr);
    a.red.counter = reinterpret_cast<unsigned*>(L->red_counter->ptr);
    a.red.result = reinterpret_cast<double*>(L->red_result->ptr);
    if (a.red.fin == FIN_NONE) a.red.fin = FIN_STORE;
  }
  const HopCost hc = hop_cost(c.prec, c.flags, c.red);
  a.site_map = c.site_map;
  a.n_map = c.n_map;
  const double bytes =
      c.count_work ? c.work_fraction * (double)L->vh * (hc.rhs_bytes * c.nrhs + hc.shared_bytes) : 0.0;
  const double flops = c.count_work ? c.work_fraction * (double)L->vh * c.nrhs * hc.rhs_flops : 0.0;
  note_launch(L, c.cls, bytes, flops, st, true);
  BR_CHECK(launch_hop_any(c.prec, c.flags, c.red, a, sh.block, st, nullptr, sh.variant), BRIDGE_EINVAL,
           "hop variant not instantiated");
  note_launch(L, c.cls, bytes, flops, st, false);
  BR_CUDA(cudaGetLastError());
}

void apply_deo(bridge_lattice_s* L, const bridge_op& op, int q, const Field& out, const Field& in, cudaStream_t st) {
  HopCall c;
  c.prec = in.prec;
  c.flags = 0;
  c.cls = K_HOP;
  c.out_parity = q;
  c.nrhs = in.nrhs;
  c.beta = -op.kappa;
  for (int k = 0; k < 4; ++k) c.bc[k] = op.bc[k];
  c.out = out.ptr(q);
  c.out_rs = out.rs;
  c.in = in.ptr(1 - q);
  c.in_rs = in.rs;
  run_hop(L, c, st);
}

void apply_d(bridge_lattice_s* L, const bridge_op& op, const Field& out, const Field& in, cudaStream_t st) {
  const bool clov = op_is_clover(op);
  for (int q = 0; q < 2; ++q) {
    HopCall c;
    c.prec = in.prec;
    c.flags = F_SELF | (clov ? F_SELF_CLOV : 0);
    c.cls = K_FULLD;
    c.out_parity = q;
    c.nrhs = in.nrhs;
    c.beta = -op.kappa;
    c.s1 = 1.0;
    c.kcsw = op_kcsw(op);
    for (int k = 0; k < 4; ++k) c.bc[k] = op.bc[k];
    c.out = out.ptr(q);
    c.out_rs = out.rs;
    c.in = in.ptr(1 - q);
    c.in_rs = in.rs;
    c.self = in.ptr(q);
    c.self_rs = in.rs;
    run_hop(L, c, st);
  }
}

void apply_dhat(bridge_lattice_s* L, const bridge_op& op, const Field& out, const Field& in, const Field& tmp,
                cudaStream_t st) {
  const bool clov = op_is_clover(op);
  HopCall c;
  c.prec = in.prec;
  c.nrhs = in.nrhs;
  c.kcsw = op_kcsw(op);
  for (int k = 0; k < 4; ++k) c.bc[k] = op.bc[k];
  // pass 1: tmp_o = T_oo^-1 (-kappa H_oe in_e)
  c.flags = clov ? F_E_CLOV : 0;
  c.cls = K_DHAT1;
  c.out_parity = 1;
  c.beta = -op.kappa;
  c.out = tmp.ptr(1);
  c.out_rs = tmp.rs;
  c.in = in.ptr(0);
  c.in_rs = in.rs;
  run_hop(L, c, st);
  // pass 2: out_e = in_e - T_ee^-1 (-kappa H_eo tmp_o)
  c.flags = F_SELF | (clov ? F_E_CLOV : 0);
  c.cls = K_DHAT2;
  c.out_parity = 0;
  c.beta = op.kappa;
  c.s1 = 1.0;
  c.out = out.ptr(0);
  c.out_rs = out.rs;
  c.in = tmp.ptr(1);
  c.in_rs = tmp.rs;
  c.self = in.ptr(0);
  c.self_rs = in.rs;
  run_hop(L, c, st);
}

// ------------------------------------------------------------ layouts
static CopyArgs copy_args(bridge_lattice_s* L, const Field& f, int parity) {
  CopyArgs a;
  std::memset(&a, 0, sizeof(a));
  a.vh = (uint32_t)L->vh;
  a.nrhs = f.nrhs;
  a.parity = parity;
  a.g = L->g;
  a.V = L->V;
  const int block = 256;
  a.nblk = (int)((L->vh + block - 1) / block);
  return a;
}

void canon_to_field(bridge_lattice_s* L, const double* canon, const Field& f, cudaStream_t st, const int* mask,
                    long canon_rs) {
  const int lo = f.subset == BRIDGE_FULL ? 0 : f.subset, hi = f.subset == BRIDGE_FULL ? 1 : f.subset;
  for (int p = lo; p <= hi; ++p) {
    CopyArgs a = copy_args(L, f, p);
    a.canon = canon;
    a.canon_rs = canon_rs / 2;
    a.canon_full = f.subset == BRIDGE_FULL;
    a.dst = f.ptr(p);
    a.dst_rs = f.rs;
    a.mask = mask;
    const double bytes = (double)L->vh * f.nrhs * (192 + spinor_site_bytes(f.prec));
    note_launch(L, K_CONVERT, bytes, 0, st, true);
    launch_canon_to_field(f.prec, a, 256, st);
    note_launch(L, K_CONVERT, bytes, 0, st, false);
  }
  BR_CUDA(cudaGetLastError());
}

void field_to_canon(bridge_lattice_s* L, const Field& f, double* canon, cudaStream_t st, long canon_rs) {
  const int lo = f.subset == BRIDGE_FULL ? 0 : f.subset, hi = f.subset == BRIDGE_FULL ? 1 : f.subset;
  for (int p = lo; p <= hi; ++p) {
    CopyArgs a = copy_args(L, f, p);
    a.canon_out = canon;
    a.canon_rs = canon_rs / 2;
    a.canon_full = f.subset == BRIDGE_FULL;
    a.src = f.ptr(p);
    a.src_rs = f.rs;
    const double bytes = (double)L->vh * f.nrhs * (192 + spinor_site_bytes(f.prec));
    note_launch(L, K_CONVERT, bytes, 0, st, true);
    launch_field_to_canon(f.prec, a, 256, st);
    note_launch(L, K_CONVERT, bytes, 0, st, false);
  }
  BR_CUDA(cudaGetLastError());
}

void convert_field(bridge_lattice_s* L, const Field& src, const Field& dst, int parity, cudaStream_t st, const int* mask) {
  CopyArgs a = copy_args(L, src, parity);
  a.src = src.ptr(parity);
  a.src_rs = src.rs;
  a.dst = dst.ptr(parity);
  a.dst_rs = dst.rs;
  a.mask = mask;
  const double bytes = (double)L->vh * src.nrhs * (spinor_site_bytes(src.prec) + spinor_site_bytes(dst.prec));
  note_launch(L, K_CONVERT, bytes, 0, st, true);
  launch_convert(src.prec, dst.prec, a, 256, st);
  note_launch(L, K_CONVERT, bytes, 0, st, false);
  BR_CUDA(cudaGetLastError());
}

void accumulate64(bridge_lattice_s* L, const Field& src, int sp, const Field& dst, int dp, cudaStream_t st,
                  const int* mask) {
  CopyArgs a = copy_args(L, src, sp);
  a.src = src.ptr(sp);
  a.src_rs = src.rs;
  a.dst = dst.ptr(dp);
  a.dst_rs = dst.rs;
  a.mask = mask;
  const double bytes = (double)L->vh * src.nrhs * (spinor_site_bytes(src.prec) + 2 * 192);
  note_launch(L, K_CONVERT, bytes, (double)L->vh * src.nrhs * 24, st, true);
  launch_accumulate64(src.prec, a, 256, st);
  note_launch(L, K_CONVERT, bytes, 0, st, false);
  BR_CUDA(cudaGetLastError());
}

void norm2_field(bridge_lattice_s* L, const Field& f, int parity, RedArgs red, cudaStream_t st) {
  CopyArgs a = copy_args(L, f, parity);
  a.src = f.ptr(parity);
  a.src_rs = f.rs;
  a.red = red;
  a.nblk = std::max(1, std::min(a.nblk, sm_count() * 8 / std::max(1, f.nrhs)));
  const double bytes = (double)L->vh * f.nrhs * spinor_site_bytes(f.prec);
  note_launch(L, K_NORM, bytes, (double)L->vh * f.nrhs * 48, st, true);
  launch_norm2(f.prec, a, 256, st);
  note_launch(L, K_NORM, bytes, 0, st, false);
  BR_CUDA(cudaGetLastError());
}

void clover_site(bridge_lattice_s* L, int prec, bool inverse, double kcsw, int parity, const Field& src, int sp,
                 const Field& dst, int dp, int nrhs, cudaStream_t st, CloverSet* set) {
  const char* cl = (set ? clover_ptr(L, *set, prec, inverse) : clover_ptr(L, prec, inverse, kcsw)) +
                   (long)parity * clover_block_bytes(prec, L->vh);
  CopyArgs a = copy_args(L, src, sp);
  a.nrhs = nrhs;
  a.src = src.ptr(sp);
  a.src_rs = src.rs;
  a.dst = dst.ptr(dp);
  a.dst_rs = dst.rs;
  const double bytes = (double)L->vh * (nrhs * 2.0 * spinor_site_bytes(prec) + clover_site_bytes(prec));
  note_launch(L, K_CLOVER, bytes, (double)L->vh * nrhs * 504, st, true);
  launch_clover_site(prec, a, cl, 256, st);
  note_launch(L, K_CLOVER, bytes, 0, st, false);
  BR_CUDA(cudaGetLastError());
}

bool hop_has_variants(int flags, int red) {
  return (flags == 0 && red == R_NONE) || (flags == F_E_CLOV && red == R_NONE) ||
         ((flags == F_SELF || flags == (F_SELF | F_E_CLOV)) && (red == R_DOT_A || red == R_TS)) ||
         (flags == (F_AUX | F_SELF | F_SELF_CLOV) && red == R_NORM);
}

bool launch_hop_any(int prec, int flags, int red, const HopArgs& a, int block, cudaStream_t st, int* occ,
                    int variant) {
  if (!hop_has_variants(flags, red)) variant = 0;
  for (;;) {
    bool ok = false;
    switch (prec) {
      case P_F64: ok = launch_hop<P_F64>(flags, red, a, block, st, occ, variant); break;
      case P_F32: ok = launch_hop<P_F32>(flags, red, a, block, st, occ, variant); break;
      case P_F16: ok = launch_hop<P_F16>(flags, red, a, block, st, occ, variant); break;
      case P_BF16: ok = launch_hop<P_BF16>(flags, red, a, block, st, occ, variant); break;
    }
    if (ok || variant == 0) return ok;
    variant = 0;  // this kernel has no such variant (e.g. several RHS per thread in FP64)
  }
}

}  // namespace bridge
