// Host-side runtime of libbridge: lattice handles, device fields, operator
// application and launch bookkeeping.  Everything here is plain C++ around
// the CUDA runtime; no PyTorch types appear.
#pragma once

#include <atomic>
#include <functional>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/bridge.h"
#include "kernels.h"

namespace bridge {

// ------------------------------------------------------------ errors
struct Error {
  int code;
  std::string msg;
};
void set_error(int code, const std::string& msg);
#define BR_CUDA(call)                                                                          \
  do {                                                                                         \
    cudaError_t e_ = (call);                                                                   \
    if (e_ != cudaSuccess) throw ::bridge::Error{BRIDGE_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)}; \
  } while (0)
#define BR_CHECK(cond, code, msg) \
  do {                            \
    if (!(cond)) throw ::bridge::Error{(code), (msg)}; \
  } while (0)

// ------------------------------------------------------- kernel stats
enum KClass {
  K_HOP = 0,     // D_eo / D_oe
  K_FULLD,       // full operator, one parity
  K_DHAT1,       // Schur pass 1: T^-1 D_oe
  K_DHAT2,       // Schur pass 2 (operator application)
  K_DHAT2A,      // Schur pass 2 with <rhat, v> -> alpha (solver)
  K_DHAT2W,      // Schur pass 2 with <t, s>, |t|^2 -> omega (solver)
  K_PREP,        // even-odd prepare / reconstruct
  K_RESID,       // FP64 residual b - D x with |r|^2
  K_BLAS_INIT,
  K_BLAS_S,
  K_BLAS_XR,
  K_BLAS_P,
  K_CONVERT,
  K_NORM,
  K_CLOVER,
  K_SETUP,
  K_DWF_MIX,       // Moebius: fifth-dimension matrix on every site
  K_DWF_HOP,       // Moebius: D_eo / D_oe and the full operator
  K_DWF_SCHUR1,    // Moebius Schur pass 1 (and of its adjoint)
  K_DWF_SCHUR2,    // Moebius Schur pass 2 (and of its adjoint)
  K_DWF_SCHUR2CG,  // adjoint pass 2 fused with the CG update of x and r
  K_DWF_PREP,      // Moebius even-odd prepare / reconstruct
  K_DWF_RESID,     // Moebius FP64 residual b - D x with |r|^2
  K_STAG_HOP,      // staggered: D_eo / D_oe and the full operator
  K_STAG_PASS1,    // staggered CG / Schur pass 1: D_oe p
  K_STAG_PASS2,    // staggered CG / Schur pass 2 with Re <p, q> -> alpha
  K_STAG_VEC,      // staggered vector kernels and conversions
  K_STAG_PREP,     // staggered even-odd prepare / reconstruct
  K_STAG_RESID,    // staggered FP64 residual with |r|^2
  K_MG_SAP,        // multigrid: SAP block minimal-residual solves
  K_MG_RESID,      // multigrid: FP32 fine residual r - D x of the smoother
  K_MG_TRANSFER,   // multigrid: restriction / prolongation
  K_MG_COARSE,     // multigrid: coarse operator applications
  K_MG_VEC,        // multigrid: vector updates and dot products (fine FP64 and coarse)
  K_MG_OUTER,      // multigrid: FP64 operator of the outer FBiCGStab
  K_MG_SETUP,      // multigrid: setup (null vectors, Gram-Schmidt, coarse operator)
  K_NCLASS
};
const char* kclass_name(int k);

struct KStat {
  long launches = 0;
  double bytes = 0, flops = 0, ms = 0;
};

// --------------------------------------------------------- device memory
// Device buffer.  With a stream, memory comes from the device's
// stream-ordered pool (cudaMallocAsync / cudaFreeAsync on that stream): no
// device-wide synchronization on release, which matters when many solves
// start and finish while others run.  Without one, plain cudaMalloc.
struct DevBuf {
  char* ptr = nullptr;
  size_t bytes = 0;
  cudaStream_t st = nullptr;
  bool async = false;
  DevBuf() = default;
  explicit DevBuf(size_t n, cudaStream_t stream = nullptr, bool stream_ordered = false);
  ~DevBuf();
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
};

// A spinor field in the GPU layout: nrhs x (1 or 2 parity blocks).
struct Field {
  int prec = P_F32;
  int subset = BRIDGE_FULL;  // BRIDGE_EVEN, BRIDGE_ODD, BRIDGE_FULL
  int nrhs = 1;
  long vh = 0;
  long block = 0;  // bytes of one parity block
  long rs = 0;     // bytes between right-hand sides
  std::shared_ptr<DevBuf> buf;
  char* ptr(int parity) const {  // block of this parity for rhs 0
    return buf->ptr + ((subset == BRIDGE_FULL && parity == 1) ? block : 0);
  }
};
Field make_field(int prec, int subset, int nrhs, long vh, cudaStream_t st = nullptr, bool stream_ordered = false);

// ----------------------------------------------------------- tuning
// Launch shapes picked per (kernel class, precision, flags, lattice, nrhs).
struct LaunchShape {
  int block = 256;
  int nblk = 0;     // site blocks per rhs; 0 -> cover the lattice once
  int variant = 0;  // register-budget variant of the kernel (see launch_hop)
};

struct Stats {
  std::mutex mu;
  KStat k[K_NCLASS];
  // optional per-launch event timing
  bool profiling = false;
  struct Rec {
    int cls;
    cudaEvent_t a, b;
  };
  std::vector<Rec> recs;
  std::vector<cudaEvent_t> pool;
};

// Clover term T = 1 - kcsw sum sigma F and its inverse for one value of
// kcsw = kappa c_sw: FP64 masters plus lazily converted copies.  Shared by
// the solves that use it, so a solve keeps its set alive even after the
// lattice cache has dropped it.
struct CloverSet {
  double kcsw = 0.0;
  std::unique_ptr<DevBuf> T[4], Tinv[4];
  std::mutex mu;
};

// Fifth-dimension matrices of one Moebius parameter set (Ls, M5, b, c, m_f):
// DWF_NMAT real [2][Ls][Ls] matrices (chirality +, then -) in FP64 and FP32.
enum DwfMat {
  DM_B = 0,     // B = b + c P
  DM_BAINV,     // B A^-1
  DM_AINV,      // A^-1
  DM_G5AINVT,   // gamma_5 A^-T
  DM_AINVTBT,   // A^-T B^T
  DM_BTG5,      // B^T gamma_5
  DM_A,         // A = (b alpha + 1) + (c alpha - 1) P
  DM_MA,        // -A
  DWF_NMAT
};
struct DwfSet {
  int Ls = 0;
  double M5 = 0, b = 0, c = 0, mf = 0;
  std::unique_ptr<DevBuf> mats[2];  // [0] FP64, [1] FP32
  SProg prog[DWF_NMAT];             // the same matrices as bidiagonal factors
  bool fact = false;                // the factored form is stable for these parameters (and not disabled)
  const void* mat(int prec, int id) const {
    const size_t per = (size_t)2 * Ls * Ls * (prec == P_F64 ? 8 : 4);
    return mats[prec == P_F64 ? 0 : 1]->ptr + id * per;
  }
};

}  // namespace bridge

// ------------------------------------------------------------- lattice
struct bridge_lattice_s {
  int dims[4];
  long V, vh;
  bridge::Geom g;
  int device = 0;
  cudaStream_t stream = nullptr;
  // links per precision; [0] (F64, 18 reals) is the master copy
  std::unique_ptr<bridge::DevBuf> gauge[4];
  bool have_gauge = false;
  // clover sets for the most recently used values of kappa * c_sw
  std::vector<std::shared_ptr<bridge::CloverSet>> clovers;
  std::mutex clover_mu;
  std::vector<std::shared_ptr<bridge::DwfSet>> dwf_sets;  // recently used Moebius parameter sets
  std::mutex dwf_mu;
  std::atomic<int> in_flight{0};  // engine requests currently holding this lattice
  // reduction scratch for the operator entry points
  std::unique_ptr<bridge::DevBuf> red_partials, red_result;
  std::unique_ptr<bridge::DevBuf> red_counter;
  double* red_result_host = nullptr;  // pinned
  // staging for canonical fields of the host-pointer entry points
  std::unique_ptr<bridge::DevBuf> stage_in, stage_out;
  std::map<std::string, bridge::LaunchShape> tuned;
  std::mutex tune_mu;
  std::map<std::string, bridge::Field> ws;  // reusable fields of the operator entry points
  bridge::Stats stats;
  std::mutex api_mu;  // serialises host entry points on one lattice
};

namespace bridge {

// launch bookkeeping (called at each launch site)
void note_launch(bridge_lattice_s* L, int cls, double bytes, double flops, cudaStream_t st, bool begin);
// Launch shape for a kernel key: the tuned entry if there is one, else
// `block` threads and a persistent grid of (resident blocks per SM x SM
// count) blocks, computed by occ(block), capped at one site per thread.
LaunchShape shape_for(bridge_lattice_s* L, const std::string& key, long vh, int nrhs,
                      const std::function<int(int)>& occ);

// Algorithmic cost of one hop launch: bytes and flops per right-hand side
// (spinors) and shared by all right-hand sides (links, clover blocks).
struct HopCost {
  double rhs_bytes, shared_bytes, rhs_flops;
};
HopCost hop_cost(int prec, int flags, int red);
int sm_count();
// Reduction scratch of the lattice's operator entry points, grown on demand.
void ensure_red_scratch(bridge_lattice_s* L, long n_partials, int nrhs);

// gauge / clover on demand
const char* gauge_ptr(bridge_lattice_s* L, int prec);
std::shared_ptr<CloverSet> clover_set(bridge_lattice_s* L, double kcsw);
const char* clover_ptr(bridge_lattice_s* L, CloverSet& set, int prec, bool inverse);
const char* clover_ptr(bridge_lattice_s* L, int prec, bool inverse, double kcsw);

// ------------------------------------------------------- operators
// Apply one hop-kernel variant (see dslash.cuh).  Field pointers are the
// parity blocks of rhs 0; strides are per right-hand side.
struct HopCall {
  int prec, flags = 0, red = R_NONE, out_parity = 0, nrhs = 1, cls = K_HOP;
  double beta = 0, s1 = 0, caux = 0;
  int bc[4] = {1, 1, 1, -1};
  char* out = nullptr;
  long out_rs = 0;
  const char *in = nullptr, *self = nullptr, *aux = nullptr, *avec = nullptr;
  long in_rs = 0, self_rs = 0, aux_rs = 0, avec_rs = 0;
  double kcsw = 0;
  CloverSet* clov = nullptr;  // optional: use this set instead of the cache lookup
  bool count_work = true;     // false: count the launch only (work is credited by the caller)
  RedArgs redargs{};
  const uint32_t* site_map = nullptr;  // HopArgs::site_map / n_map: a subset of the output sites
  uint32_t n_map = 0;
  double work_fraction = 1.0;  // share of the sites the launch computes (for the byte and flop counts)
};
void run_hop(bridge_lattice_s* L, HopCall c, cudaStream_t st);

// Operator entry points on fields (asynchronous on st).
void apply_deo(bridge_lattice_s* L, const bridge_op& op, int out_parity, const Field& out, const Field& in, cudaStream_t st);
void apply_d(bridge_lattice_s* L, const bridge_op& op, const Field& out, const Field& in, cudaStream_t st);
void apply_dhat(bridge_lattice_s* L, const bridge_op& op, const Field& out, const Field& in, const Field& tmp_odd,
                cudaStream_t st);

// Canonical FP64 (device) <-> field.  full: canonical holds whole lattices.
// canon_rs: doubles between right-hand sides of the canonical array (0: the
// field's own site count x 24, i.e. contiguous right-hand sides).
void canon_to_field(bridge_lattice_s* L, const double* canon, const Field& f, cudaStream_t st, const int* mask = nullptr,
                    long canon_rs = 0);
void field_to_canon(bridge_lattice_s* L, const Field& f, double* canon, cudaStream_t st, long canon_rs = 0);
void convert_field(bridge_lattice_s* L, const Field& src, const Field& dst, int parity, cudaStream_t st, const int* mask);
void accumulate64(bridge_lattice_s* L, const Field& src, int src_parity, const Field& dst64, int dst_parity, cudaStream_t st,
                  const int* mask);
void norm2_field(bridge_lattice_s* L, const Field& f, int parity, RedArgs red, cudaStream_t st);
void clover_site(bridge_lattice_s* L, int prec, bool inverse, double kcsw, int parity, const Field& src, int sp,
                 const Field& dst, int dp, int nrhs, cudaStream_t st, CloverSet* set = nullptr);

// Scratch data for timing runs: pseudo-random values in [-1, 1).
void fill_scratch(const Field& f, uint32_t seed, cudaStream_t st);
// Append the shape-table entries `keys` to the tuning cache file, if one is set.
void tune_cache_save(bridge_lattice_s* L, const std::vector<std::string>& keys);

// Reusable field of this lattice (allocated on first use).
Field& workspace(bridge_lattice_s* L, const std::string& name, int prec, int subset, int nrhs);

bool op_is_clover(const bridge_op& op);
double op_kcsw(const bridge_op& op);

}  // namespace bridge
