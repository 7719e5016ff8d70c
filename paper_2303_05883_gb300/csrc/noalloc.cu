// bridge_mult_Dhat_noalloc: the Schur operator applied without allocating
// any device memory during the call.
//
// Some callers cannot call cudaMalloc when they apply the operator: a host
// application that reserves all device memory up front for its own pool and
// forbids allocations afterwards, or a latency-critical loop in which
// cudaMalloc / cudaFree (which can synchronize the whole device) are not
// allowed.  This entry point serves them.  Its scratch -- the input, the odd
// intermediate and the output in the GPU site layout -- lives in one
// file-scope device array of fixed size that every GPU loading the library
// holds until the process exits.
//
// The computation is the same as bridge_mult_Dhat_dev: canonical FP64 in ->
// GPU layout, pass 1 (tmp_o = T_oo^-1 (-kappa H_oe in_e)), pass 2
// (out_e = in_e + kappa T_ee^-1 H_eo tmp_o), GPU layout -> canonical FP64.
#include <algorithm>
#include <cstring>
#include <mutex>

#include "host.h"

using namespace bridge;

namespace bridge {
extern std::atomic<long> g_launches;
}

// 64 MiB of scratch per device (three half-lattice fields of the chosen
// precision and nrhs must fit; see BRIDGE_NOALLOC_SCRATCH_BYTES in bridge.h).
static __device__ __align__(256) char g_dhat_scratch[BRIDGE_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
char* g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device (looked up once
// per device; the host-side name of the array is not a device address).
char* scratch_on_current_device() {
  int dev = 0;
  BR_CUDA(cudaGetDevice(&dev));
  BR_CHECK(dev >= 0 && dev < kMaxDevices, BRIDGE_ECUDA, "device index out of range");
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_dhat_scratch);
    if (e != cudaSuccess) {
      cudaGetLastError();
      throw Error{BRIDGE_ECUDA, std::string("cudaGetSymbolAddress of the scratch array: ") + cudaGetErrorString(e)};
    }
    g_scratch_ptr[dev] = static_cast<char*>(p);
  }
  return g_scratch_ptr[dev];
}

// Launch shape without touching the lattice's shape table: the tuned entry
// if one exists, else a persistent grid from the occupancy query.
LaunchShape shape_readonly(bridge_lattice_s* L, const std::string& key, int nrhs, const std::function<int(int)>& occ) {
  LaunchShape s;
  bool found = false;
  {
    std::lock_guard<std::mutex> lk(L->tune_mu);
    auto it = L->tuned.find(key);
    if (it != L->tuned.end()) {
      s = it->second;
      found = true;
    }
  }
  if (!found) {
    s.block = 128;
    const int per_sm = occ(s.block);
    s.nblk = std::max(1, sm_count() * (per_sm > 0 ? per_sm : 4) / std::max(1, nrhs));
  }
  const long cover = (L->vh + s.block - 1) / s.block;
  if (s.nblk <= 0 || s.nblk > cover) s.nblk = (int)cover;
  return s;
}

// The clover inverse of this lattice for kcsw in precision prec, if it was
// built before; nullptr otherwise (nothing is built here).
const char* existing_clover_inverse(bridge_lattice_s* L, double kcsw, int prec) {
  std::lock_guard<std::mutex> lk(L->clover_mu);
  for (auto& s : L->clovers)
    if (s->kcsw == kcsw) {
      std::lock_guard<std::mutex> lk2(s->mu);
      return s->Tinv[prec] ? s->Tinv[prec]->ptr : nullptr;
    }
  return nullptr;
}

}  // namespace

extern "C" int bridge_mult_Dhat_noalloc(bridge_lattice L, const bridge_op* op, int prec, const double* in_dev,
                                        double* out_dev, int nrhs) {
  try {
    BR_CHECK(L != nullptr && op != nullptr, BRIDGE_EINVAL, "NULL argument");
    BR_CHECK(prec >= BRIDGE_F64 && prec <= BRIDGE_BF16, BRIDGE_EINVAL, "precision");
    BR_CHECK(op->kind == BRIDGE_WILSON || op->kind == BRIDGE_CLOVER, BRIDGE_EINVAL, "op.kind");
    for (int k = 0; k < 4; ++k) BR_CHECK(op->bc[k] == 1 || op->bc[k] == -1, BRIDGE_EINVAL, "op.bc must be +1 or -1");
    BR_CHECK(nrhs >= 0, BRIDGE_EINVAL, "nrhs < 0");
    if (nrhs == 0) return BRIDGE_OK;
    BR_CHECK(in_dev != nullptr && out_dev != nullptr, BRIDGE_EINVAL, "in/out is NULL");
    const long block = spinor_block_bytes(prec, L->vh);
    const long need = 3L * nrhs * block;
    BR_CHECK(need <= (long)BRIDGE_NOALLOC_SCRATCH_BYTES, BRIDGE_EINVAL,
             "lattice too large for the no-allocation scratch: needs " + std::to_string(need) + " bytes, maximum " +
                 std::to_string((long)BRIDGE_NOALLOC_SCRATCH_BYTES));
    std::lock_guard<std::mutex> lk(L->api_mu);
    BR_CHECK(L->have_gauge && L->gauge[prec], BRIDGE_ESTATE,
             "links in this precision not built yet: apply the operator once with bridge_mult_Dhat first");
    const bool clov = op_is_clover(*op);
    const char* tinv = nullptr;
    if (clov) {
      tinv = existing_clover_inverse(L, op_kcsw(*op), prec);
      BR_CHECK(tinv != nullptr, BRIDGE_ESTATE,
               "clover term for this kappa*c_sw and precision not built yet: apply the operator once first");
    }
    char* scratch = scratch_on_current_device();
    char* f_in = scratch;                    // even, nrhs blocks
    char* f_tmp = scratch + nrhs * block;    // odd
    char* f_out = scratch + 2 * nrhs * block;  // even
    cudaStream_t st = L->stream;

    CopyArgs ca;
    std::memset(&ca, 0, sizeof(ca));
    ca.vh = (uint32_t)L->vh;
    ca.nrhs = nrhs;
    ca.g = L->g;
    ca.V = L->V;
    ca.nblk = (int)((L->vh + 255) / 256);
    ca.canon = in_dev;
    ca.canon_full = 0;
    ca.dst = f_in;
    ca.dst_rs = block;
    BR_CHECK(launch_canon_to_field(prec, ca, 256, st), BRIDGE_EINVAL, "precision");

    HopArgs a;
    std::memset(&a, 0, sizeof(a));
    a.g = L->g;
    a.nrhs = nrhs;
    for (int k = 0; k < 4; ++k) a.bc[k] = op->bc[k];
    a.gauge = L->gauge[prec]->ptr;
    a.clovE = tinv;
    const std::string dims = std::to_string(L->dims[0]) + "x" + std::to_string(L->dims[1]) + "x" +
                             std::to_string(L->dims[2]) + "x" + std::to_string(L->dims[3]);
    // pass 1: tmp_o = T_oo^-1 (-kappa H_oe in_e)
    const int f1 = clov ? F_E_CLOV : 0;
    a.out_parity = 1;
    a.beta = -op->kappa;
    a.out = f_tmp;
    a.out_rs = block;
    a.in = f_in;
    a.in_rs = block;
    LaunchShape s1 = shape_readonly(L, "hop/" + std::to_string(prec) + "/" + std::to_string(f1) + "/0/" + dims + "/" +
                                           std::to_string(nrhs), nrhs, [&](int b) {
      int n = 0;
      launch_hop_any(prec, f1, R_NONE, a, b, st, &n);
      return n;
    });
    a.nblk = s1.nblk;
    BR_CHECK(launch_hop_any(prec, f1, R_NONE, a, s1.block, st, nullptr, s1.variant), BRIDGE_EINVAL, "hop variant");
    // pass 2: out_e = in_e + kappa T_ee^-1 H_eo tmp_o
    const int f2 = F_SELF | (clov ? F_E_CLOV : 0);
    a.out_parity = 0;
    a.beta = op->kappa;
    a.s1 = 1.0;
    a.out = f_out;
    a.in = f_tmp;
    a.self = f_in;
    a.self_rs = block;
    LaunchShape s2 = shape_readonly(L, "hop/" + std::to_string(prec) + "/" + std::to_string(f2) + "/0/" + dims + "/" +
                                           std::to_string(nrhs), nrhs, [&](int b) {
      int n = 0;
      launch_hop_any(prec, f2, R_NONE, a, b, st, &n);
      return n;
    });
    a.nblk = s2.nblk;
    BR_CHECK(launch_hop_any(prec, f2, R_NONE, a, s2.block, st, nullptr, s2.variant), BRIDGE_EINVAL, "hop variant");

    ca.canon = nullptr;
    ca.dst = nullptr;
    ca.canon_out = out_dev;
    ca.src = f_out;
    ca.src_rs = block;
    BR_CHECK(launch_field_to_canon(prec, ca, 256, st), BRIDGE_EINVAL, "precision");
    BR_CUDA(cudaGetLastError());
    g_launches.fetch_add(4);
  } catch (const Error& e) {
    set_error(e.code, e.msg);
    return e.code;
  }
  return BRIDGE_OK;
}
