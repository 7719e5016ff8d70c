// The C-ABI of libbridge (declared in include/bridge.h): argument checks,
// host <-> device staging, and dispatch to the runtime and solver.
#include <cmath>
#include <cstring>
#include <string>

#include "dwf.h"
#include "solver.h"
#include "stag.h"

using namespace bridge;

// bridge_mult_Dhat_dag: internal selector next to bridge_apply_op
static constexpr int APPLY_DHAT_DAG = 100;

namespace bridge {
const char* last_error_text();
extern std::atomic<long> g_launches;
extern std::atomic<long> g_dev_allocs;
void tune_cache_load(bridge_lattice_s* L);
int engine_submit(bridge_lattice_s* L, const bridge_op& op, const bridge_solver& s, const double* b, int nrhs,
                  bool borrow, bridge_request_h* out);

Field& workspace(bridge_lattice_s* L, const std::string& name, int prec, int subset, int nrhs) {
  const std::string key = name + "/" + std::to_string(prec) + "/" + std::to_string(subset) + "/" + std::to_string(nrhs);
  auto it = L->ws.find(key);
  if (it != L->ws.end()) return it->second;
  return L->ws.emplace(key, make_field(prec, subset, nrhs, L->vh)).first->second;
}
}  // namespace bridge

struct bridge_field_s {
  bridge_lattice_s* L;
  Field f;
};

#define BR_API_BEGIN try {
#define BR_API_END                             \
  }                                            \
  catch (const Error& e) {                     \
    set_error(e.code, e.msg);                  \
    return e.code;                             \
  }                                            \
  catch (const std::exception& e) {            \
    set_error(BRIDGE_ENOMEM, e.what());        \
    return BRIDGE_ENOMEM;                      \
  }                                            \
  return BRIDGE_OK;

static void check_op(const bridge_op* op) {
  BR_CHECK(op != nullptr, BRIDGE_EINVAL, "op is NULL");
  BR_CHECK(op->kind == BRIDGE_WILSON || op->kind == BRIDGE_CLOVER || op->kind == BRIDGE_MOBIUS ||
               op->kind == BRIDGE_STAGGERED,
           BRIDGE_EINVAL, "op.kind");
  for (int k = 0; k < 4; ++k) BR_CHECK(op->bc[k] == 1 || op->bc[k] == -1, BRIDGE_EINVAL, "op.bc must be +1 or -1");
  if (op->kind == BRIDGE_MOBIUS)
    check_mobius(*op);
  else if (op->kind == BRIDGE_STAGGERED)
    check_staggered(*op);
  else
    BR_CHECK(std::isfinite(op->kappa) && std::isfinite(op->csw), BRIDGE_EINVAL, "op.kappa / op.csw not finite");
}
// Entry points that serve only some operator kinds.
static void check_not_mobius(const bridge_op* op, const char* what) {
  BR_CHECK(op->kind != BRIDGE_MOBIUS, BRIDGE_EINVAL, std::string(what) + " does not take MOBIUS operators");
}
static void check_not_staggered(const bridge_op* op, const char* what) {
  BR_CHECK(op->kind != BRIDGE_STAGGERED, BRIDGE_EINVAL, std::string(what) + " does not take STAGGERED operators");
}
// Doubles per site of one right-hand side of a canonical spinor argument.
static long site_doubles(const bridge_op& op) {
  return op.kind == BRIDGE_MOBIUS ? 24L * op.Ls : op.kind == BRIDGE_STAGGERED ? 6L : 24L;
}
static void check_prec(int prec) {
  BR_CHECK(prec >= BRIDGE_F64 && prec <= BRIDGE_BF16, BRIDGE_EINVAL, "precision");
}
static void check_lat(bridge_lattice L, bool need_gauge) {
  BR_CHECK(L != nullptr, BRIDGE_EINVAL, "lattice is NULL");
  if (need_gauge) BR_CHECK(L->have_gauge, BRIDGE_ESTATE, "no gauge field uploaded");
}

static char* stage(std::unique_ptr<DevBuf>& b, size_t n) {
  if (!b || b->bytes < n) {
    b.reset();
    b.reset(new DevBuf(n));
  }
  return b->ptr;
}

// ---------------------------------------------------------------- operators
static void mult_dev(bridge_lattice_s* L, const bridge_op& op, int prec, int which, int out_parity, const double* in,
                     double* out, int nrhs) {
  cudaStream_t st = L->stream;
  if (op_is_staggered(op)) {
    BR_CHECK(prec == BRIDGE_F64 || prec == BRIDGE_F32, BRIDGE_EINVAL, "STAGGERED operators run in F64 or F32");
    BR_CHECK(which != APPLY_DHAT_DAG, BRIDGE_EINVAL, "bridge_mult_Dhat_dag is provided for MOBIUS operators only");
    if (which == BRIDGE_APPLY_D) {
      Field& fi = stag_workspace(L, "mult_in", prec, BRIDGE_FULL, nrhs);
      Field& fo = stag_workspace(L, "mult_out", prec, BRIDGE_FULL, nrhs);
      stag_canon_to_field(L, in, fi, true, st);
      stag_apply_d(L, op, fo, fi, st);
      stag_field_to_canon(L, fo, out, true, st);
    } else if (which == BRIDGE_APPLY_DEO) {
      const int q = out_parity;
      Field& fi = stag_workspace(L, "mult_in", prec, 1 - q, nrhs);
      Field& fo = stag_workspace(L, "mult_out", prec, q, nrhs);
      stag_canon_to_field(L, in, fi, false, st);
      stag_apply_deo(L, op, q, fo, fi, st);
      stag_field_to_canon(L, fo, out, false, st);
    } else {
      Field& fi = stag_workspace(L, "mult_in", prec, BRIDGE_EVEN, nrhs);
      Field& fo = stag_workspace(L, "mult_out", prec, BRIDGE_EVEN, nrhs);
      stag_canon_to_field(L, in, fi, false, st);
      stag_apply_dhat(L, op, fo, fi, st);
      stag_field_to_canon(L, fo, out, false, st);
    }
    return;
  }
  if (op_is_mobius(op)) {
    BR_CHECK(prec == BRIDGE_F64 || prec == BRIDGE_F32, BRIDGE_EINVAL, "MOBIUS operators run in F64 or F32");
    const int nq = nrhs * op.Ls;
    if (which == BRIDGE_APPLY_D) {
      Field& fi = workspace(L, "mult_in", prec, BRIDGE_FULL, nq);
      Field& fo = workspace(L, "mult_out", prec, BRIDGE_FULL, nq);
      canon_to_field(L, in, fi, st);
      dwf_apply_d(L, op, fo, fi, st);
      field_to_canon(L, fo, out, st);
    } else if (which == BRIDGE_APPLY_DEO) {
      const int q = out_parity;
      Field& fi = workspace(L, "mult_in", prec, 1 - q, nq);
      Field& fo = workspace(L, "mult_out", prec, q, nq);
      canon_to_field(L, in, fi, st);
      dwf_apply_deo(L, op, q, fo, fi, st);
      field_to_canon(L, fo, out, st);
    } else {
      Field& fi = workspace(L, "mult_in", prec, BRIDGE_EVEN, nq);
      Field& fo = workspace(L, "mult_out", prec, BRIDGE_EVEN, nq);
      canon_to_field(L, in, fi, st);
      dwf_apply_dhat(L, op, fo, fi, which == APPLY_DHAT_DAG, st);
      field_to_canon(L, fo, out, st);
    }
    return;
  }
  BR_CHECK(which != APPLY_DHAT_DAG, BRIDGE_EINVAL, "bridge_mult_Dhat_dag is provided for MOBIUS operators only");
  if (which == BRIDGE_APPLY_D) {
    Field& fi = workspace(L, "mult_in", prec, BRIDGE_FULL, nrhs);
    Field& fo = workspace(L, "mult_out", prec, BRIDGE_FULL, nrhs);
    canon_to_field(L, in, fi, st);
    apply_d(L, op, fo, fi, st);
    field_to_canon(L, fo, out, st);
  } else if (which == BRIDGE_APPLY_DEO) {
    const int q = out_parity;
    Field& fi = workspace(L, "mult_in", prec, 1 - q, nrhs);
    Field& fo = workspace(L, "mult_out", prec, q, nrhs);
    canon_to_field(L, in, fi, st);
    apply_deo(L, op, q, fo, fi, st);
    field_to_canon(L, fo, out, st);
  } else {
    Field& fi = workspace(L, "mult_in", prec, BRIDGE_EVEN, nrhs);
    Field& fo = workspace(L, "mult_out", prec, BRIDGE_EVEN, nrhs);
    Field& ft = workspace(L, "mult_tmp", prec, BRIDGE_ODD, nrhs);
    canon_to_field(L, in, fi, st);
    apply_dhat(L, op, fo, fi, ft, st);
    field_to_canon(L, fo, out, st);
  }
}

static int mult_common(bridge_lattice L, const bridge_op* op, int prec, int which, int out_parity, const double* in,
                       double* out, int nrhs, bool host) {
  BR_API_BEGIN
  check_lat(L, true);
  check_op(op);
  check_prec(prec);
  BR_CHECK(out_parity == 0 || out_parity == 1, BRIDGE_EINVAL, "out_parity must be 0 or 1");
  BR_CHECK(nrhs >= 0, BRIDGE_EINVAL, "nrhs < 0");
  if (nrhs == 0) return BRIDGE_OK;
  BR_CHECK(in != nullptr && out != nullptr, BRIDGE_EINVAL, "in/out is NULL");
  std::lock_guard<std::mutex> lk(L->api_mu);
  const long sites = which == BRIDGE_APPLY_D ? L->V : L->vh;
  const size_t n = (size_t)nrhs * site_doubles(*op) * sites * sizeof(double);
  if (host) {
    double* din = reinterpret_cast<double*>(stage(L->stage_in, n));
    double* dout = reinterpret_cast<double*>(stage(L->stage_out, n));
    BR_CUDA(cudaMemcpyAsync(din, in, n, cudaMemcpyHostToDevice, L->stream));
    mult_dev(L, *op, prec, which, out_parity, din, dout, nrhs);
    BR_CUDA(cudaMemcpyAsync(out, dout, n, cudaMemcpyDeviceToHost, L->stream));
    BR_CUDA(cudaStreamSynchronize(L->stream));
  } else {
    mult_dev(L, *op, prec, which, out_parity, in, out, nrhs);
  }
  BR_API_END
}

// ------------------------------------------------------------------ solver
static int solve_common(bridge_lattice L, const bridge_op* op, const bridge_solver* s, const double* b, double* x,
                        int nrhs, bridge_info* info, bool host) {
  BR_API_BEGIN
  check_lat(L, true);
  check_op(op);
  BR_CHECK(s != nullptr, BRIDGE_EINVAL, "solver params NULL");
  BR_CHECK(s->tol > 0 && std::isfinite(s->tol), BRIDGE_EINVAL, "tol must be > 0");
  if (s->mixed) check_prec(s->inner_prec);
  BR_CHECK(nrhs >= 0, BRIDGE_EINVAL, "nrhs < 0");
  if (nrhs == 0) return BRIDGE_OK;
  BR_CHECK(b != nullptr && x != nullptr, BRIDGE_EINVAL, "b/x is NULL");
  std::lock_guard<std::mutex> lk(L->api_mu);
  const size_t n = (size_t)nrhs * site_doubles(*op) * L->V * sizeof(double);
  const double* db = b;
  double* dx = x;
  if (host) {
    db = reinterpret_cast<double*>(stage(L->stage_in, n));
    dx = reinterpret_cast<double*>(stage(L->stage_out, n));
    BR_CUDA(cudaMemcpyAsync(const_cast<double*>(db), b, n, cudaMemcpyHostToDevice, L->stream));
    BR_CUDA(cudaMemcpyAsync(dx, x, n, cudaMemcpyHostToDevice, L->stream));
  }
  int status;
  if (op_is_mobius(*op)) {
    status = dwf_solve(L, *op, *s, db, dx, nrhs, info);
  } else if (op_is_staggered(*op)) {
    status = stag_solve(L, *op, *s, db, dx, nrhs, info);
  } else {
    SolveState S(L, *op, *s, nrhs, L->stream, db, dx);
    while (!S.advance()) BR_CUDA(cudaEventSynchronize(S.wait_event()));
    if (info)
      for (int r = 0; r < nrhs; ++r) info[r] = S.info()[r];
    status = S.status();
  }
  if (host) {
    BR_CUDA(cudaMemcpyAsync(x, dx, n, cudaMemcpyDeviceToHost, L->stream));
    BR_CUDA(cudaStreamSynchronize(L->stream));
  }
  if (status != BRIDGE_OK) set_error(status, "solver did not reach tolerance");
  return status;
  BR_API_END
}

extern "C" {

int bridge_lattice_create(const int dims[4], bridge_lattice* out) {
  BR_API_BEGIN
  BR_CHECK(dims != nullptr && out != nullptr, BRIDGE_EINVAL, "NULL argument");
  *out = nullptr;
  long V = 1;
  for (int k = 0; k < 4; ++k) {
    BR_CHECK(dims[k] >= 2 && dims[k] % 2 == 0, BRIDGE_EINVAL, "extents must be even and >= 2");
    V *= dims[k];
  }
  BR_CHECK(V / 2 < (1L << 31), BRIDGE_EINVAL, "lattice too large (V/2 >= 2^31)");
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    throw Error{BRIDGE_ECUDA, std::string("no CUDA device: ") + cudaGetErrorString(e)};
  }
  int dev = 0;
  BR_CUDA(cudaGetDevice(&dev));
  cudaDeviceProp prop;
  BR_CUDA(cudaGetDeviceProperties(&prop, dev));
  BR_CHECK(prop.major == 10 && prop.minor == 3, BRIDGE_ECUDA,
           std::string("libbridge is built for sm_103a only; device is sm_") + std::to_string(prop.major) +
               std::to_string(prop.minor));
  auto* L = new bridge_lattice_s();
  for (int k = 0; k < 4; ++k) L->dims[k] = dims[k];
  L->V = V;
  L->vh = V / 2;
  L->g = make_geom(dims);
  L->device = dev;
  cudaError_t se = cudaStreamCreateWithFlags(&L->stream, cudaStreamNonBlocking);
  if (se != cudaSuccess) {
    delete L;
    throw Error{BRIDGE_ECUDA, cudaGetErrorString(se)};
  }
  tune_cache_load(L);
  *out = L;
  BR_API_END
}

int bridge_lattice_destroy(bridge_lattice L) {
  BR_API_BEGIN
  if (!L) return BRIDGE_OK;
  BR_CHECK(L->in_flight.load() == 0, BRIDGE_ESTATE, "requests on this lattice are still running");
  cudaStreamSynchronize(L->stream);
  {
    std::lock_guard<std::mutex> lk(L->stats.mu);
    for (auto& r : L->stats.recs) {
      cudaEventDestroy(r.a);
      cudaEventDestroy(r.b);
    }
    for (auto e : L->stats.pool) cudaEventDestroy(e);
  }
  cudaStream_t st = L->stream;
  delete L;
  cudaStreamDestroy(st);
  BR_API_END
}

void* bridge_lattice_stream(bridge_lattice L) { return L ? (void*)L->stream : nullptr; }

int bridge_sync(bridge_lattice L) {
  BR_API_BEGIN
  check_lat(L, false);
  BR_CUDA(cudaStreamSynchronize(L->stream));
  BR_API_END
}

static int gauge_upload(bridge_lattice L, const double* U, const bridge_op* op, bool host) {
  BR_API_BEGIN
  check_lat(L, false);
  BR_CHECK(U != nullptr, BRIDGE_EINVAL, "U is NULL");
  if (op) check_op(op);
  std::lock_guard<std::mutex> lk(L->api_mu);
  const size_t n = (size_t)4 * L->V * 18 * sizeof(double);
  const double* src = U;
  if (host) {
    char* d = stage(L->stage_in, n);
    BR_CUDA(cudaMemcpyAsync(d, U, n, cudaMemcpyHostToDevice, L->stream));
    src = reinterpret_cast<const double*>(d);
  }
  BR_CHECK(L->in_flight.load() == 0, BRIDGE_ESTATE, "requests on this lattice are still running");
  BR_CUDA(cudaStreamSynchronize(L->stream));
  for (int p = 0; p < 4; ++p) L->gauge[p].reset();
  {
    std::lock_guard<std::mutex> lk(L->clover_mu);
    L->clovers.clear();
  }
  L->gauge[P_F64].reset(new DevBuf((size_t)(8 * link_block_bytes(P_F64, L->vh))));
  note_launch(L, K_SETUP, (double)n * 2, 0, L->stream, true);
  launch_gauge_from_canon(src, L->g, L->gauge[P_F64]->ptr, L->stream);
  note_launch(L, K_SETUP, 0, 0, L->stream, false);
  BR_CUDA(cudaGetLastError());
  L->have_gauge = true;
  if (op && op_is_clover(*op)) {
    clover_ptr(L, P_F64, true, op_kcsw(*op));
  }
  BR_CUDA(cudaStreamSynchronize(L->stream));
  if (host) L->stage_in.reset();  // the link staging buffer is as large as the FP64 links
  BR_API_END
}

int bridge_gauge_upload(bridge_lattice L, const double* U, const bridge_op* op) { return gauge_upload(L, U, op, true); }
int bridge_gauge_upload_dev(bridge_lattice L, const double* U, const bridge_op* op) {
  return gauge_upload(L, U, op, false);
}

int bridge_mult_D(bridge_lattice L, const bridge_op* op, int prec, const double* in, double* out, int nrhs) {
  return mult_common(L, op, prec, BRIDGE_APPLY_D, 0, in, out, nrhs, true);
}
int bridge_mult_Deo(bridge_lattice L, const bridge_op* op, int prec, int out_parity, const double* in, double* out,
                    int nrhs) {
  return mult_common(L, op, prec, BRIDGE_APPLY_DEO, out_parity, in, out, nrhs, true);
}
int bridge_mult_Dhat(bridge_lattice L, const bridge_op* op, int prec, const double* in, double* out, int nrhs) {
  return mult_common(L, op, prec, BRIDGE_APPLY_DHAT, 0, in, out, nrhs, true);
}
int bridge_mult_Dhat_dag(bridge_lattice L, const bridge_op* op, int prec, const double* in, double* out, int nrhs) {
  return mult_common(L, op, prec, APPLY_DHAT_DAG, 0, in, out, nrhs, true);
}
int bridge_mult_Dhat_dag_dev(bridge_lattice L, const bridge_op* op, int prec, const double* in, double* out,
                             int nrhs) {
  return mult_common(L, op, prec, APPLY_DHAT_DAG, 0, in, out, nrhs, false);
}
int bridge_mult_D_dev(bridge_lattice L, const bridge_op* op, int prec, const double* in, double* out, int nrhs) {
  return mult_common(L, op, prec, BRIDGE_APPLY_D, 0, in, out, nrhs, false);
}
int bridge_mult_Deo_dev(bridge_lattice L, const bridge_op* op, int prec, int out_parity, const double* in, double* out,
                        int nrhs) {
  return mult_common(L, op, prec, BRIDGE_APPLY_DEO, out_parity, in, out, nrhs, false);
}
int bridge_mult_Dhat_dev(bridge_lattice L, const bridge_op* op, int prec, const double* in, double* out, int nrhs) {
  return mult_common(L, op, prec, BRIDGE_APPLY_DHAT, 0, in, out, nrhs, false);
}

void bridge_solver_defaults(bridge_solver* s) {
  if (!s) return;
  std::memset(s, 0, sizeof(*s));
  s->tol = 1e-10;
  s->max_iter = 20000;
  s->inner_prec = BRIDGE_F32;
  s->inner_tol = 0.0;
  s->mixed = 1;
  s->check_every = 16;
  s->use_graph = 1;
  s->max_outer = 50;
  s->method = BRIDGE_METHOD_AUTO;
}

int bridge_solve(bridge_lattice L, const bridge_op* op, const bridge_solver* s, const double* b, double* x, int nrhs,
                 bridge_info* info) {
  return solve_common(L, op, s, b, x, nrhs, info, true);
}
int bridge_solve_dev(bridge_lattice L, const bridge_op* op, const bridge_solver* s, const double* b, double* x,
                     int nrhs, bridge_info* info) {
  return solve_common(L, op, s, b, x, nrhs, info, false);
}

// ------------------------------------------------------------------ fields
int bridge_field_create(bridge_lattice L, int prec, int subset, int nrhs, bridge_field* out) {
  BR_API_BEGIN
  check_lat(L, false);
  check_prec(prec);
  BR_CHECK(out != nullptr, BRIDGE_EINVAL, "out is NULL");
  BR_CHECK(subset >= BRIDGE_EVEN && subset <= BRIDGE_FULL, BRIDGE_EINVAL, "subset");
  BR_CHECK(nrhs >= 1, BRIDGE_EINVAL, "nrhs must be >= 1");
  auto* f = new bridge_field_s();
  f->L = L;
  try {
    f->f = make_field(prec, subset, nrhs, L->vh);
  } catch (...) {
    delete f;
    throw;
  }
  *out = f;
  BR_API_END
}

int bridge_field_destroy(bridge_field f) {
  BR_API_BEGIN
  if (!f) return BRIDGE_OK;
  cudaStreamSynchronize(f->L->stream);
  delete f;
  BR_API_END
}

static size_t canon_bytes(const bridge_field_s* f) {
  const long sites = f->f.subset == BRIDGE_FULL ? f->L->V : f->L->vh;
  return (size_t)f->f.nrhs * sites * 24 * sizeof(double);
}

int bridge_field_import(bridge_field f, const double* src, int on_device) {
  BR_API_BEGIN
  BR_CHECK(f != nullptr && src != nullptr, BRIDGE_EINVAL, "NULL argument");
  bridge_lattice_s* L = f->L;
  std::lock_guard<std::mutex> lk(L->api_mu);
  const double* d = src;
  if (!on_device) {
    const size_t n = canon_bytes(f);
    char* s = stage(L->stage_in, n);
    BR_CUDA(cudaMemcpyAsync(s, src, n, cudaMemcpyHostToDevice, L->stream));
    d = reinterpret_cast<const double*>(s);
  }
  canon_to_field(L, d, f->f, L->stream);
  if (!on_device) BR_CUDA(cudaStreamSynchronize(L->stream));
  BR_API_END
}

int bridge_field_export(bridge_field f, double* dst, int on_device) {
  BR_API_BEGIN
  BR_CHECK(f != nullptr && dst != nullptr, BRIDGE_EINVAL, "NULL argument");
  bridge_lattice_s* L = f->L;
  std::lock_guard<std::mutex> lk(L->api_mu);
  if (on_device) {
    field_to_canon(L, f->f, dst, L->stream);
  } else {
    const size_t n = canon_bytes(f);
    double* s = reinterpret_cast<double*>(stage(L->stage_out, n));
    field_to_canon(L, f->f, s, L->stream);
    BR_CUDA(cudaMemcpyAsync(dst, s, n, cudaMemcpyDeviceToHost, L->stream));
    BR_CUDA(cudaStreamSynchronize(L->stream));
  }
  BR_API_END
}

int bridge_apply(bridge_lattice L, const bridge_op* op, int which, bridge_field out, bridge_field in) {
  BR_API_BEGIN
  check_lat(L, true);
  check_op(op);
  BR_CHECK(out != nullptr && in != nullptr, BRIDGE_EINVAL, "NULL field");
  BR_CHECK(out->L == L && in->L == L, BRIDGE_EINVAL, "field belongs to another lattice");
  BR_CHECK(out->f.prec == in->f.prec, BRIDGE_EINVAL, "fields differ in precision");
  BR_CHECK(out->f.nrhs == in->f.nrhs, BRIDGE_EINVAL, "fields differ in nrhs");
  BR_CHECK(out->f.buf != in->f.buf, BRIDGE_EINVAL, "in and out must differ");
  std::lock_guard<std::mutex> lk(L->api_mu);
  check_not_staggered(op, "bridge_apply");
  if (op_is_mobius(*op)) {
    BR_CHECK(in->f.nrhs % op->Ls == 0, BRIDGE_EINVAL, "MOBIUS fields hold a multiple of Ls slices");
    BR_CHECK(in->f.prec == BRIDGE_F64 || in->f.prec == BRIDGE_F32, BRIDGE_EINVAL, "MOBIUS operators run in F64 or F32");
    switch (which) {
      case BRIDGE_APPLY_D:
        BR_CHECK(in->f.subset == BRIDGE_FULL && out->f.subset == BRIDGE_FULL, BRIDGE_EINVAL, "D needs FULL fields");
        dwf_apply_d(L, *op, out->f, in->f, L->stream);
        break;
      case BRIDGE_APPLY_DEO:
      case BRIDGE_APPLY_DOE: {
        const int q = which == BRIDGE_APPLY_DEO ? 0 : 1;
        BR_CHECK(in->f.subset != q && out->f.subset != 1 - q, BRIDGE_EINVAL, "hopping block maps between parities");
        dwf_apply_deo(L, *op, q, out->f, in->f, L->stream);
        break;
      }
      case BRIDGE_APPLY_DHAT:
        BR_CHECK(in->f.subset != BRIDGE_ODD && out->f.subset != BRIDGE_ODD, BRIDGE_EINVAL, "D^ acts on even fields");
        dwf_apply_dhat(L, *op, out->f, in->f, false, L->stream);
        break;
      default:
        throw Error{BRIDGE_EINVAL, "unknown operator"};
    }
    return BRIDGE_OK;
  }
  switch (which) {
    case BRIDGE_APPLY_D:
      BR_CHECK(in->f.subset == BRIDGE_FULL && out->f.subset == BRIDGE_FULL, BRIDGE_EINVAL, "D needs FULL fields");
      apply_d(L, *op, out->f, in->f, L->stream);
      break;
    case BRIDGE_APPLY_DEO:
      BR_CHECK(in->f.subset != BRIDGE_EVEN && out->f.subset != BRIDGE_ODD, BRIDGE_EINVAL, "D_eo maps odd to even");
      apply_deo(L, *op, 0, out->f, in->f, L->stream);
      break;
    case BRIDGE_APPLY_DOE:
      BR_CHECK(in->f.subset != BRIDGE_ODD && out->f.subset != BRIDGE_EVEN, BRIDGE_EINVAL, "D_oe maps even to odd");
      apply_deo(L, *op, 1, out->f, in->f, L->stream);
      break;
    case BRIDGE_APPLY_DHAT: {
      BR_CHECK(in->f.subset != BRIDGE_ODD && out->f.subset != BRIDGE_ODD, BRIDGE_EINVAL, "D^ acts on even fields");
      Field& tmp = workspace(L, "apply_tmp", in->f.prec, BRIDGE_ODD, in->f.nrhs);
      apply_dhat(L, *op, out->f, in->f, tmp, L->stream);
      break;
    }
    default:
      throw Error{BRIDGE_EINVAL, "unknown operator"};
  }
  BR_API_END
}

// ------------------------------------------------------------- diagnostics
const char* bridge_strerror(int s) {
  switch (s) {
    case BRIDGE_OK: return "ok";
    case BRIDGE_PENDING: return "pending";
    case BRIDGE_EINVAL: return "invalid argument";
    case BRIDGE_ENOMEM: return "out of device memory or over budget";
    case BRIDGE_ENOCONV: return "solver did not converge";
    case BRIDGE_EBREAKDOWN: return "solver breakdown";
    case BRIDGE_ETIMEDOUT: return "timed out";
    case BRIDGE_ECUDA: return "CUDA error";
    case BRIDGE_ESTATE: return "call out of order";
  }
  return "unknown status";
}

const char* bridge_last_error(void) { return last_error_text(); }

int bridge_stats(bridge_lattice L, bridge_kstat* out, int n) {
  if (!L) return BRIDGE_EINVAL;
  std::lock_guard<std::mutex> lk(L->stats.mu);
  if (!L->stats.recs.empty()) {
    for (auto& r : L->stats.recs) {
      float ms = 0.f;
      if (cudaEventSynchronize(r.b) == cudaSuccess && cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess)
        L->stats.k[r.cls].ms += ms;
      else
        cudaGetLastError();
      L->stats.pool.push_back(r.a);
      L->stats.pool.push_back(r.b);
    }
    L->stats.recs.clear();
  }
  for (int k = 0; k < n && k < K_NCLASS; ++k) {
    out[k].name = kclass_name(k);
    out[k].launches = L->stats.k[k].launches;
    out[k].bytes = L->stats.k[k].bytes;
    out[k].flops = L->stats.k[k].flops;
    out[k].ms = L->stats.k[k].ms;
  }
  return K_NCLASS;
}

int bridge_stats_reset(bridge_lattice L) {
  if (!L) return BRIDGE_EINVAL;
  bridge_kstat tmp[K_NCLASS];
  bridge_stats(L, tmp, K_NCLASS);
  std::lock_guard<std::mutex> lk(L->stats.mu);
  for (auto& k : L->stats.k) k = KStat{};
  return BRIDGE_OK;
}

int bridge_profile(bridge_lattice L, int enable) {
  if (!L) return BRIDGE_EINVAL;
  std::lock_guard<std::mutex> lk(L->stats.mu);
  L->stats.profiling = enable != 0;
  return BRIDGE_OK;
}

long bridge_launch_count(void) { return g_launches.load(); }
long bridge_device_alloc_count(void) { return g_dev_allocs.load(); }

int bridge_debug_neighbours(const int dims[4], int parity, long ih, long out[8], int wraps[8]) {
  BR_API_BEGIN
  BR_CHECK(dims && out && wraps, BRIDGE_EINVAL, "NULL argument");
  for (int k = 0; k < 4; ++k) BR_CHECK(dims[k] >= 2 && dims[k] % 2 == 0, BRIDGE_EINVAL, "extents");
  Geom g = make_geom(dims);
  BR_CHECK(ih >= 0 && ih < (long)g.vh && (parity == 0 || parity == 1), BRIDGE_EINVAL, "site");
  int c[4];
  uint32_t xh;
  site_coords(g, (uint32_t)ih, parity, c, xh);
  uint32_t f, b;
  bool wf, wb;
  neighbours<0>(g, (uint32_t)ih, c, xh, f, b, wf, wb);
  out[0] = f; out[1] = b; wraps[0] = wf; wraps[1] = wb;
  neighbours<1>(g, (uint32_t)ih, c, xh, f, b, wf, wb);
  out[2] = f; out[3] = b; wraps[2] = wf; wraps[3] = wb;
  neighbours<2>(g, (uint32_t)ih, c, xh, f, b, wf, wb);
  out[4] = f; out[5] = b; wraps[4] = wf; wraps[5] = wb;
  neighbours<3>(g, (uint32_t)ih, c, xh, f, b, wf, wb);
  out[6] = f; out[7] = b; wraps[6] = wf; wraps[7] = wb;
  BR_API_END
}

static int submit(bridge_lattice L, const bridge_op* op, const bridge_solver* s, const double* b, int nrhs,
                  bool borrow, bridge_request_h* out) {
  BR_API_BEGIN
  check_lat(L, true);
  check_op(op);
  check_not_mobius(op, "bridge_submit");
  check_not_staggered(op, "bridge_submit");
  BR_CHECK(s != nullptr && b != nullptr && out != nullptr, BRIDGE_EINVAL, "NULL argument");
  BR_CHECK(s->tol > 0, BRIDGE_EINVAL, "tol must be > 0");
  if (s->mixed) check_prec(s->inner_prec);
  BR_CHECK(nrhs >= 1, BRIDGE_EINVAL, "nrhs must be >= 1");
  return engine_submit(L, *op, *s, b, nrhs, borrow, out);
  BR_API_END
}

int bridge_submit(bridge_lattice L, const bridge_op* op, const bridge_solver* s, const double* b, int nrhs,
                  bridge_request_h* out) {
  return submit(L, op, s, b, nrhs, false, out);
}

int bridge_submit_borrowed(bridge_lattice L, const bridge_op* op, const bridge_solver* s, const double* b, int nrhs,
                           bridge_request_h* out) {
  return submit(L, op, s, b, nrhs, true, out);
}

}  // extern "C"
