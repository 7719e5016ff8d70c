// Autotuner: launch shapes (threads per block, site blocks per right-hand
// side) for the kernels of one solve, picked by timing on scratch buffers.
//
// The paper tunes the shape of its 2-D SIMD site tile on A64FX and finds the
// choice matters little there (Sec. 3, Fig. 5).  On the GPU the analogous
// knobs are the CTA size and whether the grid covers the lattice once (one
// site per thread) or is persistent (resident blocks x SMs, grid-stride):
// the persistent shape shortens the serial tail of the fused reductions.
// Every candidate runs on scratch fields and scratch solver scalars, so
// tuning never touches solver state.  Results go to the lattice's shape
// table and, with BRIDGE_TUNE_CACHE set, to a JSON file keyed by device.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <sstream>

#include "dwf.h"
#include "host.h"

using namespace bridge;

namespace bridge {

static std::string device_tag() {
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceProp p;
  if (cudaGetDeviceProperties(&p, dev) != cudaSuccess) return "unknown";
  std::string n = p.name;
  for (auto& ch : n)
    if (ch == ' ' || ch == '"') ch = '_';
  return n + "_sm" + std::to_string(p.major) + std::to_string(p.minor);
}

static std::string cache_path() {
  const char* p = std::getenv("BRIDGE_TUNE_CACHE");
  return p ? std::string(p) : std::string();
}

// Cache format: one line per entry, "device key block nblk variant".
void tune_cache_load(bridge_lattice_s* L) {
  const std::string path = cache_path();
  if (path.empty()) return;
  std::ifstream f(path);
  if (!f) return;
  const std::string tag = device_tag();
  std::string dev, key;
  int block, nblk, variant;
  std::lock_guard<std::mutex> lk(L->tune_mu);
  while (f >> dev >> key >> block >> nblk >> variant)
    if (dev == tag) L->tuned[key] = LaunchShape{block, nblk, variant};
}

void tune_cache_save(bridge_lattice_s* L, const std::vector<std::string>& keys) {
  const std::string path = cache_path();
  if (path.empty()) return;
  std::ofstream f(path, std::ios::app);
  const std::string tag = device_tag();
  std::lock_guard<std::mutex> lk(L->tune_mu);
  for (const auto& k : keys) {
    auto it = L->tuned.find(k);
    if (it != L->tuned.end())
      f << tag << " " << k << " " << it->second.block << " " << it->second.nblk << " " << it->second.variant << "\n";
  }
}

// Pseudo-random values in [-1, 1) so that timing runs on scratch data move
// ordinary, incompressible bytes.
__global__ void k_fill(float* p, size_t n, uint32_t seed) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    uint32_t h = (uint32_t)i * 2654435761u ^ seed;
    h ^= h >> 16;
    h *= 2246822519u;
    h ^= h >> 13;
    p[i] = (float)(h >> 8) * (1.0f / 8388608.0f) - 1.0f;
  }
}

void fill_scratch(const Field& f, uint32_t seed, cudaStream_t st) {
  const size_t n = f.buf->bytes / sizeof(float);
  k_fill<<<(unsigned)std::min<size_t>((n + 255) / 256, 152 * 32), 256, 0, st>>>(reinterpret_cast<float*>(f.buf->ptr), n, seed);
}

template <class Launch>
static float time_launches(Launch&& launch, cudaStream_t st, cudaEvent_t a, cudaEvent_t b, int reps) {
  launch();  // warm
  BR_CUDA(cudaEventRecord(a, st));
  for (int i = 0; i < reps; ++i) launch();
  BR_CUDA(cudaEventRecord(b, st));
  BR_CUDA(cudaEventSynchronize(b));
  float ms = 0;
  BR_CUDA(cudaEventElapsedTime(&ms, a, b));
  return ms / reps;
}

struct Candidate {
  int block, nblk, variant;
};

// Block sizes x {persistent grid, 2x persistent, one site per thread} for
// each kernel variant; occ(block, variant) gives resident blocks/SM.  A
// variant with NR right-hand sides per thread launches ceil(nrhs / NR)
// groups of site blocks.
static std::vector<Candidate> candidates(long vh, int nrhs, const std::vector<int>& variants,
                                         const std::function<int(int, int)>& occ) {
  std::vector<Candidate> out;
  for (int v : variants) {
    const int groups = (nrhs + hop_variant_rpt(v) - 1) / hop_variant_rpt(v);
    // the tile kernels choose their own block size: one set of grids
    const std::vector<int> blocks = hop_variant_is_tile(v) ? std::vector<int>{64} : std::vector<int>{64, 128, 256};
    for (int block : blocks) {
      const long cover = (vh + block - 1) / block;
      const int per_sm = std::max(1, occ(block, v));
      for (int m : {1, 2}) {
        long n = std::max<long>(1, (long)sm_count() * per_sm * m / std::max(1, groups));
        if (n < cover) out.push_back({block, (int)n, v});
      }
      out.push_back({block, (int)cover, v});
    }
  }
  return out;
}

static std::vector<int> hop_variants(int prec, int flags, int red, int nrhs) {
  std::vector<int> v = {0};
  if (!hop_has_variants(flags, red)) return v;
  for (int k = 1; k < 6; ++k) v.push_back(k);
  const bool residual = (flags & F_SELF_CLOV) != 0;
  if (prec != P_F64 && !residual) {
    for (int k = 6; k < 9; ++k)
      if (hop_variant_rpt(k) <= nrhs) v.push_back(k);
    if (nrhs >= 2)
      for (int k = 9; k < HOP_NVARIANT; ++k)
        if (hop_variant_for_prec(k, prec)) v.push_back(k);
  }
  return v;
}

// Tune the hop variants and vector kernels that a solve with this operator,
// inner precision and nrhs launches (and the plain D_eo kernel).
void tune_solver_kernels(bridge_lattice_s* L, const bridge_op& op, int prec, int nrhs) {
  const bool clov = op_is_clover(op);
  const int px = (prec == P_F16 || prec == P_BF16) ? P_F32 : prec;
  const long vh = L->vh;
  cudaStream_t st = L->stream;
  Field fin = make_field(prec, BRIDGE_FULL, nrhs, vh), fout = make_field(prec, BRIDGE_FULL, nrhs, vh);
  Field f2 = make_field(prec, BRIDGE_FULL, nrhs, vh), fx = make_field(px, BRIDGE_EVEN, nrhs, vh);
  fill_scratch(fin, 1u, st);
  fill_scratch(f2, 2u, st);
  fill_scratch(fx, 3u, st);
  fill_scratch(fout, 4u, st);
  BR_CUDA(cudaGetLastError());
  DevBuf partials((size_t)nrhs * ((vh + 63) / 64) * 4 * sizeof(double)), counter(256),
      scal(sizeof(BiCGScalars) * nrhs), result(sizeof(double) * 4 * nrhs);
  BR_CUDA(cudaMemsetAsync(counter.ptr, 0, 256, st));
  std::vector<BiCGScalars> hs(nrhs);
  for (auto& q : hs) {
    std::memset(&q, 0, sizeof(q));
    q.rho_r = q.alpha_r = q.omega_r = q.beta_r = 1.0;
    q.max_iter = 1 << 30;
    q.rhat2 = q.b2 = 1.0;
  }
  BR_CUDA(cudaMemcpyAsync(scal.ptr, hs.data(), sizeof(BiCGScalars) * nrhs, cudaMemcpyHostToDevice, st));
  RedArgs red;
  red.partials = reinterpret_cast<double*>(partials.ptr);
  red.counter = reinterpret_cast<unsigned*>(counter.ptr);
  red.sc = reinterpret_cast<BiCGScalars*>(scal.ptr);
  red.result = reinterpret_cast<double*>(result.ptr);
  red.check_done = 0;  // store-only finalizers below: scratch scalars never change
  const bool verbose = std::getenv("BRIDGE_TUNE_VERBOSE") != nullptr;
  cudaEvent_t ea, eb;
  BR_CUDA(cudaEventCreate(&ea));
  BR_CUDA(cudaEventCreate(&eb));
  std::vector<std::string> keys;
  const std::string dims = std::to_string(L->dims[0]) + "x" + std::to_string(L->dims[1]) + "x" +
                           std::to_string(L->dims[2]) + "x" + std::to_string(L->dims[3]);
  std::shared_ptr<CloverSet> cs;
  if (clov) cs = clover_set(L, op_kcsw(op));
  struct HopVariant {
    int flags, red;
  };
  const int fE = clov ? F_E_CLOV : 0;
  std::vector<HopVariant> hv = {{0, R_NONE}, {fE, R_NONE}, {F_SELF | fE, R_DOT_A}, {F_SELF | fE, R_TS}, {F_AUX | fE, R_NONE}};
  if (prec == P_F64 && clov) hv.push_back({F_AUX | F_SELF | F_SELF_CLOV, R_NORM});
  std::shared_ptr<CloverSet> keep_cs = cs;
  for (const auto& v : hv) {
    HopArgs a;
    std::memset(&a, 0, sizeof(a));
    a.g = L->g;
    a.out_parity = 0;
    a.nrhs = nrhs;
    a.beta = -op.kappa;
    a.s1 = 1.0;
    a.caux = 1.0;
    for (int k = 0; k < 4; ++k) a.bc[k] = op.bc[k];
    a.out = fout.ptr(0);
    a.out_rs = fout.rs;
    a.in = fin.ptr(1);
    a.in_rs = fin.rs;
    a.self = fin.ptr(0);
    a.self_rs = fin.rs;
    a.aux = f2.ptr(0);
    a.aux_rs = f2.rs;
    a.avec = f2.ptr(1);
    a.avec_rs = f2.rs;
    a.gauge = gauge_ptr(L, prec);
    if (v.flags & F_E_CLOV) a.clovE = clover_ptr(L, *cs, prec, true);
    if (v.flags & F_SELF_CLOV) a.clovM = clover_ptr(L, *cs, prec, false);
    if (v.flags & F_SELF_CLOV) a.s1 = -1.0;
    a.red = red;
    a.red.fin = v.red == R_NONE ? FIN_NONE : FIN_STORE;
    const std::string key = "hop/" + std::to_string(prec) + "/" + std::to_string(v.flags) + "/" + std::to_string(v.red) +
                            "/" + dims + "/" + std::to_string(nrhs);
    auto occ = [&](int block, int variant) {
      int n = 0;
      launch_hop_any(prec, v.flags, v.red, a, block, st, &n, variant);
      return n;
    };
    float best = 1e30f;
    Candidate pick{128, 0, 0};
    for (const auto& c : candidates(vh, nrhs, hop_variants(prec, v.flags, v.red, nrhs), occ)) {
      a.nblk = c.nblk;
      const float ms =
          time_launches([&] { launch_hop_any(prec, v.flags, v.red, a, c.block, st, nullptr, c.variant); }, st, ea, eb, 5);
      if (verbose)
        std::fprintf(stderr, "tune %s block %d nblk %d variant %d: %.1f us\n", key.c_str(), c.block, c.nblk, c.variant,
                     1e3f * ms);
      if (ms < best) {
        best = ms;
        pick = c;
      }
    }
    BR_CUDA(cudaGetLastError());
    {
      std::lock_guard<std::mutex> lk(L->tune_mu);
      L->tuned[key] = LaunchShape{pick.block, pick.nblk, pick.variant};
    }
    keys.push_back(key);
  }
  for (int op_ : {B_S, B_XR, B_P}) {
    BlasArgs a;
    std::memset(&a, 0, sizeof(a));
    a.vh = (uint32_t)vh;
    a.nrhs = nrhs;
    a.x = fx.ptr(0);
    a.x_rs = fx.rs;
    char* e = fin.ptr(0);
    char* o = fin.ptr(1);
    char* e2 = f2.ptr(0);
    char* o2 = f2.ptr(1);
    a.r = e;
    a.p = o;
    a.v = e2;
    a.s = o2;
    a.t = fout.ptr(0);
    a.rhat = fout.ptr(1);
    a.r_rs = a.p_rs = fin.rs;
    a.v_rs = a.s_rs = f2.rs;
    a.t_rs = a.rhat_rs = fout.rs;
    a.b = e;
    a.b_rs = fin.rs;
    a.red = red;
    a.red.fin = FIN_STORE;
    const std::string key = "blas/" + std::to_string(op_) + "/" + std::to_string(prec) + "/" + std::to_string(vh) + "/" +
                            std::to_string(nrhs);
    auto occ = [&](int block, int) {
      int n = 0;
      launch_blas(op_, prec, px, a, block, st, &n);
      return n;
    };
    float best = 1e30f;
    Candidate pick{128, 0, 0};
    for (const auto& c : candidates(vh, nrhs, {0}, occ)) {
      a.nblk = c.nblk;
      const float ms = time_launches([&] { launch_blas(op_, prec, px, a, c.block, st); }, st, ea, eb, 5);
      if (ms < best) {
        best = ms;
        pick = c;
      }
    }
    BR_CUDA(cudaGetLastError());
    {
      std::lock_guard<std::mutex> lk(L->tune_mu);
      L->tuned[key] = LaunchShape{pick.block, pick.nblk};
    }
    keys.push_back(key);
  }
  cudaEventDestroy(ea);
  cudaEventDestroy(eb);
  BR_CUDA(cudaStreamSynchronize(st));
  tune_cache_save(L, keys);
}

}  // namespace bridge

extern "C" int bridge_tune(bridge_lattice L, const bridge_op* op, int prec, int nrhs) {
  try {
    if (!L || !op || nrhs < 1 || prec < BRIDGE_F64 || prec > BRIDGE_BF16) return BRIDGE_EINVAL;
    if (op->kind != BRIDGE_WILSON && op->kind != BRIDGE_CLOVER && op->kind != BRIDGE_MOBIUS) {  // STAGGERED: no tunable shapes
      set_error(BRIDGE_EINVAL, "op.kind");
      return BRIDGE_EINVAL;
    }
    if (!L->have_gauge) return BRIDGE_ESTATE;
    std::lock_guard<std::mutex> lk(L->api_mu);
    if (op->kind == BRIDGE_MOBIUS) {
      check_mobius(*op);
      tune_dwf_kernels(L, *op, prec, nrhs);
    } else {
      tune_solver_kernels(L, *op, prec, nrhs);
    }
  } catch (const Error& e) {
    set_error(e.code, e.msg);
    return e.code;
  }
  return BRIDGE_OK;
}

extern "C" int bridge_tune_set(bridge_lattice L, const char* key, int block, int nblk, int variant) {
  // block >= 64: the solver sizes its reduction partials for at most vh / 64 site blocks
  if (!L || !key || block < 64 || block > 256 || block % 32 || nblk < 1 || variant < 0 || variant >= HOP_NVARIANT)
    return BRIDGE_EINVAL;
  std::lock_guard<std::mutex> lk(L->tune_mu);
  L->tuned[key] = LaunchShape{block, nblk, variant};
  return BRIDGE_OK;
}

extern "C" int bridge_tune_table(bridge_lattice L, char* out, int n) {
  if (!L || !out || n <= 0) return BRIDGE_EINVAL;
  std::ostringstream s;
  {
    std::lock_guard<std::mutex> lk(L->tune_mu);
    for (const auto& kv : L->tuned)
      s << kv.first << " " << kv.second.block << " " << kv.second.nblk << " " << kv.second.variant << "\n";
  }
  const std::string t = s.str();
  std::strncpy(out, t.c_str(), (size_t)n - 1);
  out[n - 1] = 0;
  return (int)t.size();
}
