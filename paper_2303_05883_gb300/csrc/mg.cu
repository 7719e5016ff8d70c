// Two-level multigrid for the clover operator (host side and small kernels).
//
// Sec. 3 of the paper: outer Flexible BiCGStab with a single-precision
// two-level preconditioner (DD-alpha-AMG variant), SAP smoother with
// fixed-step minimal-residual block solves, BiCGStab on the coarse grid,
// 16 or 24 null vectors.  Here:
//   setup   null vectors v_i ~ D^-1 eta_i (mixed-precision solves of random
//           sources to a loose tolerance, i.e. one step of inverse iteration),
//           or vectors the caller passes; Gram-Schmidt per aggregate;
//           D_c = P^dag D P from probes: for every basis column (chirality,
//           vector) the block-local operator D_B and the eight single-hop
//           couplings across block faces, each restricted to the aggregates;
//   cycle   e_c = BiCGStab(D_c, P^dag r) to a loose tolerance; z = P e_c;
//           SAP cycles on the remaining residual (post-smoothing), FP32;
//   solve   FP64 defect correction around FP32 FBiCGStab passes on D with the
//           cycle as the preconditioner (the paper's outer FBiCGStab with a
//           single-precision preconditioner, with the outer iteration itself
//           in FP32 between FP64 true residuals).
// The scalars of the coarse BiCGStab and of the outer solver live on the
// host: each of their iterations costs one preconditioner cycle or one coarse
// operator application, far more than the reads of the scalars.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <vector>

#include "mg.cuh"
#include "solver.h"

namespace bridge {
namespace {

__global__ void k_mg_random(double* p, long n, uint32_t seed) {
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    uint32_t h = (uint32_t)i * 2654435761u ^ (seed * 0x9e3779b9u);
    h ^= h >> 16;
    h *= 2246822519u;
    h ^= h >> 13;
    h *= 3266489917u;
    h ^= h >> 16;
    p[i] = (double)(h >> 8) * (1.0 / 8388608.0) - 1.0;
  }
}

// w = v with the components of the other chirality zeroed (full FP32 fields).
__global__ void k_mg_chiral(const float4* v, float4* w, long n_planes_sites, long per_chi, int chi) {
  // each parity block: 6 float4 planes of vh sites; planes 0-2 hold spins
  // 0, 1 (chirality +), planes 3-5 spins 2, 3
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n_planes_sites; i += (long)gridDim.x * blockDim.x) {
    const bool keep = (i / per_chi) == chi;  // first three planes: chirality +
    w[i] = keep ? v[i] : make_float4(0.f, 0.f, 0.f, 0.f);
  }
}

// Dc[X][mode][col][row] = tmp[X][row]
__global__ void k_mg_scatter_column(const float2* tmp, float2* Dc, int nblocks, int n2, int mode, int col) {
  const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long)nblocks * n2) return;
  const int X = (int)(t / n2), row = (int)(t % n2);
  Dc[(((long)X * 9 + mode) * n2 + col) * n2 + row] = tmp[t];
}

// FP16 copy of Dc[m][col][row] (m = X * 9 + d); with tiled != 0 in the
// layout coarse_row_h4 reads, out[((m * (n2 / 4) + col / 4) * n2 + row) * 4 + col % 4].
__global__ void k_mg_to_half(const float2* in, __half2* out, long nmat, int n2, int tiled) {
  const long n = nmat * n2 * n2;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    long src = i;
    if (tiled) {
      const int j = (int)(i % 4);
      long t = i / 4;
      const int row = (int)(t % n2);
      t /= n2;
      const int g = (int)(t % (n2 / 4));
      const long m = t / (n2 / 4);
      src = (m * n2 + 4 * g + j) * n2 + row;
    }
    out[i] = __float22half2_rn(in[src]);
  }
}

unsigned grid_for(long n, int threads = 256) {
  return (unsigned)std::max<long>(1, std::min<long>((n + threads - 1) / threads, (long)sm_count() * 16));
}

}  // namespace
}  // namespace bridge

using namespace bridge;

struct bridge_mg_s {
  bridge_lattice_s* L = nullptr;
  bridge_op op{};
  bridge_mg_params prm{};
  MgGeom m{};
  int nv = 0, n2 = 0;
  long nc = 0;  // complex numbers in a coarse vector
  std::shared_ptr<CloverSet> clov;
  Field V;  // nv FP32 full fields
  std::unique_ptr<DevBuf> Dc, Dch, cvec, partial;  // Dch: FP16 copy of Dc for the coarse solver
  std::unique_ptr<DevBuf> Deo;  // FP16 tiles of the even-odd coarse system (null: solve the full system)
  std::unique_ptr<DevBuf> cnbr;                     // [nblocks][9] coarse neighbours
  std::unique_ptr<PinnedBuf> hpart;
  // coarse BiCGStab: scalars, reduction partials and ticket counter
  std::unique_ptr<DevBuf> csc, cpart, ccount;
  std::unique_ptr<PinnedBuf> hcsc;
  long coarse_iters = 0, coarse_solves = 0;
  int last_coarse_iters = 0;  // iterations of the previous coarse solve (sizes the first batch)
  Field r32, x32, res32;  // fine FP32 work fields of the cycle
  int sap_clover_smem = 1;  // SAP kernel variant (picked by timing at setup)
  bool sap_fused = true;    // residual formed inside the SAP sweep (BRIDGE_MG_SAP_FUSED=0: separate pass)
  // half-lattice sites of parity p in blocks of colour c: smap[soff[p][c] .. + sn[p][c])
  std::unique_ptr<DevBuf> smap;
  long soff[2][2] = {{0, 0}, {0, 0}}, sn[2][2] = {{0, 0}, {0, 0}};
  // error word of the streamed coarse kernel, in the scalar buffer after the BiCGScalars
  int* cerr() const { return reinterpret_cast<int*>(static_cast<char*>(csc->ptr) + 192); }
  float2* cv(int k) const { return reinterpret_cast<float2*>(cvec->ptr) + (long)k * nc; }
};

namespace bridge {
namespace {

cudaStream_t stream_of(const bridge_mg_s* g) { return g->L->stream; }

// ---- flat complex vectors (coarse float2, fine FP64 double2 per parity block)
template <class T>
void vaxpy(bridge_mg_s* g, long n, cx<double> a, const T* x, cx<double> b, T* y, cx<double> c, const T* z) {
  using S = decltype(T{}.x);
  const double bytes = (double)n * sizeof(T) * (2 + (b.r != 0 || b.i != 0 ? 1 : 0) + (z ? 1 : 0));
  note_launch(g->L, K_MG_VEC, bytes, 0, stream_of(g), true);
  mg_axpbypcz_kernel<T, S><<<grid_for(n), 256, 0, stream_of(g)>>>(n, cx<S>{(S)a.r, (S)a.i}, x, cx<S>{(S)b.r, (S)b.i},
                                                                   y, cx<S>{(S)c.r, (S)c.i}, z);
  note_launch(g->L, K_MG_VEC, bytes, 0, stream_of(g), false);
  BR_CUDA(cudaGetLastError());
}

// Every dot product launches exactly 1024 blocks (grid-stride), so each
// slot's 1024 partial sums are all written.
template <class T>
void vdot_launch(bridge_mg_s* g, long n, const T* x, const T* y, int slot) {
  const unsigned grid = 1024;
  note_launch(g->L, K_MG_VEC, (double)n * 2 * sizeof(T), 0, stream_of(g), true);
  mg_dot_kernel<T><<<grid, 256, 0, stream_of(g)>>>(n, x, y, reinterpret_cast<double2*>(g->partial->ptr) + slot * 1024);
  note_launch(g->L, K_MG_VEC, (double)n * 2 * sizeof(T), 0, stream_of(g), false);
  BR_CUDA(cudaGetLastError());
}

// Sum of the partials of `slots` dot products (fixed order); blocks the host.
std::vector<cx<double>> vdot_collect(bridge_mg_s* g, int slots) {
  BR_CUDA(cudaMemcpyAsync(g->hpart->ptr, g->partial->ptr, sizeof(double2) * 1024 * slots, cudaMemcpyDeviceToHost,
                          stream_of(g)));
  BR_CUDA(cudaStreamSynchronize(stream_of(g)));
  const double2* h = static_cast<const double2*>(g->hpart->ptr);
  std::vector<cx<double>> out(slots, cx<double>{0.0, 0.0});
  for (int s = 0; s < slots; ++s)
    for (int k = 0; k < 1024; ++k) out[s] = out[s] + cx<double>{h[s * 1024 + k].x, h[s * 1024 + k].y};
  return out;
}

// ---- fine FP64 full fields as two flat segments
long fine_n(const Field& f) { return 12L * f.vh; }
// ---- transfer and coarse operator
MgTransferArgs transfer_args(bridge_mg_s* g) {
  MgTransferArgs a;
  std::memset(static_cast<void*>(&a), 0, sizeof(a));
  a.m = g->m;
  a.nv = g->nv;
  a.V = g->V.ptr(0);
  a.V_rs = g->V.rs;
  a.field_block = g->V.block;
  return a;
}
unsigned block_threads(const bridge_mg_s* g) { return (unsigned)((g->m.bsites + 31) / 32 * 32); }

void restrict_to(bridge_mg_s* g, const Field& fine, float2* out) {
  MgTransferArgs a = transfer_args(g);
  a.fine_in = fine.ptr(0);
  a.coarse_out = out;
  const double bytes = (double)g->L->V * 96 * (1 + g->nv) + g->nc * 8.0;
  note_launch(g->L, K_MG_TRANSFER, bytes, 0, stream_of(g), true);
  mg_restrict_kernel<<<g->m.nblocks, block_threads(g), 0, stream_of(g)>>>(a);
  note_launch(g->L, K_MG_TRANSFER, bytes, 0, stream_of(g), false);
  BR_CUDA(cudaGetLastError());
}
void prolong_to(bridge_mg_s* g, const float2* c, const Field& fine, bool add) {
  MgTransferArgs a = transfer_args(g);
  a.fine_out = fine.ptr(0);
  a.coarse_in = c;
  a.add = add ? 1 : 0;
  const double bytes = (double)g->L->V * 96 * (1 + g->nv + (add ? 1 : 0)) + g->nc * 8.0;
  note_launch(g->L, K_MG_TRANSFER, bytes, 0, stream_of(g), true);
  mg_prolong_kernel<<<g->m.nblocks, block_threads(g), 0, stream_of(g)>>>(a);
  note_launch(g->L, K_MG_TRANSFER, bytes, 0, stream_of(g), false);
  BR_CUDA(cudaGetLastError());
}
template <int RED>
void launch_coarse_red(int n2, const MgCoarseArgs& a, unsigned grid, cudaStream_t st) {
  // row lengths of 4, 8, 12, 16 and 24 null vectors (mg_coarse_unrolled) unroll at compile time
  switch (n2) {
    case 8: mg_coarse_kernel<RED, 8><<<grid, 256, 0, st>>>(a); break;
    case 16: mg_coarse_kernel<RED, 16><<<grid, 256, 0, st>>>(a); break;
    case 24: mg_coarse_kernel<RED, 24><<<grid, 256, 0, st>>>(a); break;
    case 32: mg_coarse_kernel<RED, 32><<<grid, 256, 0, st>>>(a); break;
    case 48: mg_coarse_kernel<RED, 48><<<grid, 256, 0, st>>>(a); break;
    default: mg_coarse_kernel<RED, 0><<<grid, 256, 0, st>>>(a); break;
  }
}
// The streamed FP16 kernel: `stages` tile buffers (2 .. 4, up to ~70 KB
// unless two tiles are larger), a persistent grid of up to 4 CTAs per SM as
// shared memory allows.
template <int RED, int N2>
void launch_coarse_tma_n(MgCoarseArgs a, int nblocks, cudaStream_t st) {
  constexpr long tile = mg_coarse_tile_bytes<N2>();
  a.stages = (int)std::max(2L, std::min(4L, 70L * 1024 / tile));
  const long smem = a.stages * tile;
  static std::mutex mu;
  static std::map<int, long> done;
  int dev = 0;
  BR_CUDA(cudaGetDevice(&dev));
  {
    std::lock_guard<std::mutex> lock(mu);
    if (done[dev] < smem) {
      BR_CUDA(cudaFuncSetAttribute(mg_coarse_tma_kernel<RED, N2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)smem));
      done[dev] = smem;
    }
  }
  const long per_sm = std::max(1L, std::min(4L, (220L * 1024) / (smem + 4 * 1024)));
  const long grid = std::min<long>(nblocks, per_sm * sm_count());
  mg_coarse_tma_kernel<RED, N2><<<(unsigned)grid, 256, (size_t)smem, st>>>(a);
}
template <int RED>
void launch_coarse_tma(int n2, const MgCoarseArgs& a, int nblocks, cudaStream_t st) {
  switch (n2) {
    case 8: launch_coarse_tma_n<RED, 8>(a, nblocks, st); break;
    case 16: launch_coarse_tma_n<RED, 16>(a, nblocks, st); break;
    case 24: launch_coarse_tma_n<RED, 24>(a, nblocks, st); break;
    case 32: launch_coarse_tma_n<RED, 32>(a, nblocks, st); break;
    default: launch_coarse_tma_n<RED, 48>(a, nblocks, st); break;
  }
}
// Blocks of the streamed kernel at most (sizes the reduction partials).
long coarse_tma_max_grid() { return 4L * sm_count(); }

void launch_coarse(int red, int n2, const MgCoarseArgs& a, unsigned grid, cudaStream_t st) {
  if (red == MG_CR_ALPHA) launch_coarse_red<MG_CR_ALPHA>(n2, a, grid, st);
  else if (red == MG_CR_OMEGA) launch_coarse_red<MG_CR_OMEGA>(n2, a, grid, st);
  else launch_coarse_red<MG_CR_NONE>(n2, a, grid, st);
}

// Polls of each site-loop wait of the streamed kernel: the full bound, or
// BRIDGE_MG_WAIT_POLLS from the environment (read at every launch), which
// lets a test make those waits give up and exercise the error path.
static int coarse_wait_polls() {
  const char* e = std::getenv("BRIDGE_MG_WAIT_POLLS");
  if (!e || !*e) return MG_WAIT_POLLS;
  const long v = std::strtol(e, nullptr, 10);
  return (int)std::max(0L, std::min<long>(v, MG_WAIT_POLLS));
}

// Clear the streamed kernel's error word before a coarse solve or apply.
static void clear_coarse_err(bridge_mg_s* g) {
  BR_CUDA(cudaMemsetAsync(g->cerr(), 0, sizeof(int), stream_of(g)));
}

// One streamed application of the FP16 tiles T (Dch: D_c; Deo: the even-odd
// pieces): y = sum_{d0 <= d < d1} T[X][d] x_Y (or b - sum) at the coarse
// sites of one colour (parity -1: every site), with an optional fused
// reduction for the coarse BiCGStab.
void coarse_stream(bridge_mg_s* g, const DevBuf& tiles, int parity, int d0, int d1, const float2* x, float2* y,
                   const float2* b, int red, const float2* rhat, const float2* xin) {
  MgCoarseArgs a;
  std::memset(static_cast<void*>(&a), 0, sizeof(a));
  a.m = g->m;
  a.n2 = g->n2;
  a.Dch = reinterpret_cast<const __half2*>(tiles.ptr);
  a.nbr = reinterpret_cast<const int*>(g->cnbr->ptr);
  a.err = g->cerr();
  a.wait_polls = coarse_wait_polls();
  a.x = x;
  a.b = b;
  a.y = y;
  a.rhat = rhat;
  a.xin = xin;
  a.parity = parity;
  a.d0 = d0;
  a.d1 = d1;
  if (red != MG_CR_NONE) {
    a.red.partials = reinterpret_cast<double*>(g->cpart->ptr);
    a.red.counter = reinterpret_cast<unsigned*>(g->ccount->ptr);
    a.red.sc = reinterpret_cast<BiCGScalars*>(g->csc->ptr);
    a.red.fin = red == MG_CR_ALPHA ? FIN_ALPHA : FIN_OMEGA;
    a.red.check_done = 1;
  }
  const int sites = parity < 0 ? g->m.nblocks : g->m.nblocks / 2;
  const double nsite = (double)sites * g->n2;
  const double bytes = (double)sites * (d1 - d0) * g->n2 * g->n2 * 4 +
                       8.0 * nsite * (2 + (b ? 1 : 0) + (red != MG_CR_NONE ? 1 : 0));
  note_launch(g->L, K_MG_COARSE, bytes, (double)sites * (d1 - d0) * g->n2 * g->n2 * 8, stream_of(g), true);
  if (red == MG_CR_ALPHA)
    launch_coarse_tma<MG_CR_ALPHA>(g->n2, a, sites, stream_of(g));
  else if (red == MG_CR_OMEGA)
    launch_coarse_tma<MG_CR_OMEGA>(g->n2, a, sites, stream_of(g));
  else
    launch_coarse_tma<MG_CR_NONE>(g->n2, a, sites, stream_of(g));
  note_launch(g->L, K_MG_COARSE, bytes, 0, stream_of(g), false);
  BR_CUDA(cudaGetLastError());
}

void coarse_apply(bridge_mg_s* g, const float2* x, float2* y, const float2* b = nullptr, int red = MG_CR_NONE,
                  const float2* rhat = nullptr, bool half = false) {
  if (half && g->Dch && mg_coarse_unrolled(g->n2)) {  // the tiled FP16 copy: streamed by bulk copies
    coarse_stream(g, *g->Dch, -1, 0, 9, x, y, b, red, rhat, nullptr);
    return;
  }
  MgCoarseArgs a;
  std::memset(static_cast<void*>(&a), 0, sizeof(a));
  a.m = g->m;
  a.n2 = g->n2;
  a.Dc = reinterpret_cast<const float2*>(g->Dc->ptr);
  a.Dch = (half && g->Dch) ? reinterpret_cast<const __half2*>(g->Dch->ptr) : nullptr;
  a.nbr = reinterpret_cast<const int*>(g->cnbr->ptr);
  a.x = x;
  a.b = b;
  a.y = y;
  a.rhat = rhat;
  if (red != MG_CR_NONE) {
    a.red.partials = reinterpret_cast<double*>(g->cpart->ptr);
    a.red.counter = reinterpret_cast<unsigned*>(g->ccount->ptr);
    a.red.sc = reinterpret_cast<BiCGScalars*>(g->csc->ptr);
    a.red.fin = red == MG_CR_ALPHA ? FIN_ALPHA : FIN_OMEGA;
    a.red.check_done = 1;
  }
  const long n = g->nc;
  const double bytes = (double)g->m.nblocks * 9 * g->n2 * g->n2 * (a.Dch ? 4 : 8) + n * 8.0 * (b ? 3 : 2);
  note_launch(g->L, K_MG_COARSE, bytes, (double)g->m.nblocks * 9 * g->n2 * g->n2 * 8, stream_of(g), true);
  launch_coarse(red, g->n2, a, (unsigned)((n + 255) / 256), stream_of(g));
  note_launch(g->L, K_MG_COARSE, bytes, 0, stream_of(g), false);
  BR_CUDA(cudaGetLastError());
}

static_assert(sizeof(BiCGScalars) <= 192, "the coarse error word follows the scalars");

// The host copy of the scalar buffer (hcsc) holds the streamed coarse
// kernel's error word at byte 192.
void check_coarse_err(bridge_mg_s* g) {
  const int e = *reinterpret_cast<const int*>(static_cast<const char*>(g->hcsc->ptr) + 192);
  if (e == 1) throw Error{BRIDGE_ECUDA, "coarse operator: a tile copy did not complete within its wait bound"};
  if (e != 0)
    throw Error{BRIDGE_ECUDA,
                "coarse operator: a tile copy did not complete within its wait bound, and copies still in flight "
                "did not land before the kernel returned; the CUDA context is no longer reliable"};
}

void cbicg_step(bridge_mg_s* g, int op, const float2* b = nullptr) {
  MgCBicgArgs a;
  std::memset(static_cast<void*>(&a), 0, sizeof(a));
  a.n = g->nc;
  a.x = g->cv(1);
  a.r = g->cv(2);
  a.rhat = g->cv(3);
  a.p = g->cv(4);
  a.v = g->cv(5);
  a.s = g->cv(6);
  a.t = g->cv(7);
  a.b = b;
  a.red.partials = reinterpret_cast<double*>(g->cpart->ptr);
  a.red.counter = reinterpret_cast<unsigned*>(g->ccount->ptr);
  a.red.sc = reinterpret_cast<BiCGScalars*>(g->csc->ptr);
  a.red.fin = op == MG_CB_INIT ? FIN_INIT : op == MG_CB_XR ? FIN_RHO : FIN_NONE;
  a.red.check_done = op == MG_CB_INIT ? 0 : 1;
  const unsigned grid = (unsigned)std::min<long>((g->nc + 255) / 256, 2L * sm_count());
  const double bytes = (double)g->nc * 8 * (op == MG_CB_INIT ? 6 : op == MG_CB_S ? 3 : op == MG_CB_XR ? 8 : 4);
  note_launch(g->L, K_MG_VEC, bytes, 0, stream_of(g), true);
  switch (op) {
    case MG_CB_INIT: mg_cbicg_kernel<MG_CB_INIT><<<grid, 256, 0, stream_of(g)>>>(a); break;
    case MG_CB_S: mg_cbicg_kernel<MG_CB_S><<<grid, 256, 0, stream_of(g)>>>(a); break;
    case MG_CB_XR: mg_cbicg_kernel<MG_CB_XR><<<grid, 256, 0, stream_of(g)>>>(a); break;
    default: mg_cbicg_kernel<MG_CB_P><<<grid, 256, 0, stream_of(g)>>>(a); break;
  }
  note_launch(g->L, K_MG_VEC, bytes, 0, stream_of(g), false);
  BR_CUDA(cudaGetLastError());
}

// ---- coarse BiCGStab: D_c e = r to a relative tolerance, the scalars on the
// device (the van der Vorst recurrences of reduce.cuh); the host polls the
// done flag every `batch` iterations.  Solution in cv(1).
int coarse_solve(bridge_mg_s* g, const float2* rhs) {
  cudaStream_t st = stream_of(g);
  BiCGScalars init;
  std::memset(&init, 0, sizeof(init));
  init.tol2 = g->prm.coarse_tol * g->prm.coarse_tol;
  init.max_iter = std::max(1, g->prm.coarse_maxiter);
  init.rho_r = init.alpha_r = init.omega_r = 1.0;
  BR_CUDA(cudaMemcpyAsync(g->csc->ptr, &init, sizeof(init), cudaMemcpyHostToDevice, st));
  clear_coarse_err(g);
  const bool eo = g->Deo != nullptr;
  if (eo) {
    // even-odd: cv8 = A_O^-1 r_O; cv10 = A_E^-1 r_E - (A^-1 H)_EO cv8 (zero on O),
    // the right-hand side of the even system; t (cv7) stays zero on O
    const DevBuf& T = *g->Deo;
    BR_CUDA(cudaMemsetAsync(g->cv(10), 0, sizeof(float2) * g->nc, st));
    BR_CUDA(cudaMemsetAsync(g->cv(7), 0, sizeof(float2) * g->nc, st));
    coarse_stream(g, T, 1, 0, 1, rhs, g->cv(8), nullptr, MG_CR_NONE, nullptr, nullptr);
    coarse_stream(g, T, 0, 0, 1, rhs, g->cv(10), nullptr, MG_CR_NONE, nullptr, nullptr);
    coarse_stream(g, T, 0, 1, 9, g->cv(8), g->cv(10), g->cv(10), MG_CR_NONE, nullptr, nullptr);
  }
  cbicg_step(g, MG_CB_INIT, eo ? g->cv(10) : rhs);
  // The first batch runs to just short of the previous solve's count without
  // a host poll; later batches are short.  Iterations queued past
  // convergence exit at once (their kernels check the done flag).
  int batch = std::max(4, g->last_coarse_iters - 2);
  int launched = 0;
  for (;; batch = 4) {
    for (int k = 0; k < batch && launched < g->prm.coarse_maxiter; ++k, ++launched) {
      if (eo) {  // the operator 1 - (A^-1 H)_EO (A^-1 H)_OE on E, in two streamed passes
        const DevBuf& T = *g->Deo;
        coarse_stream(g, T, 1, 1, 9, g->cv(4), g->cv(9), nullptr, MG_CR_NONE, nullptr, nullptr);
        coarse_stream(g, T, 0, 1, 9, g->cv(9), g->cv(5), g->cv(4), MG_CR_ALPHA, g->cv(3), nullptr);  // v, alpha
        cbicg_step(g, MG_CB_S);                                                                   // s
        coarse_stream(g, T, 1, 1, 9, g->cv(6), g->cv(9), nullptr, MG_CR_NONE, nullptr, nullptr);
        coarse_stream(g, T, 0, 1, 9, g->cv(9), g->cv(7), g->cv(6), MG_CR_OMEGA, nullptr, g->cv(6));  // t, omega
      } else {
        coarse_apply(g, g->cv(4), g->cv(5), nullptr, MG_CR_ALPHA, g->cv(3), true);  // v = D_c p, alpha
        cbicg_step(g, MG_CB_S);                                                    // s = r - alpha v
        coarse_apply(g, g->cv(6), g->cv(7), nullptr, MG_CR_OMEGA, nullptr, true);  // t = D_c s, omega
      }
      cbicg_step(g, MG_CB_XR);  // x, r; rho, beta
      cbicg_step(g, MG_CB_P);   // p
    }
    BR_CUDA(cudaMemcpyAsync(g->hcsc->ptr, g->csc->ptr, 256, cudaMemcpyDeviceToHost, st));
    BR_CUDA(cudaStreamSynchronize(st));
    check_coarse_err(g);
    const BiCGScalars* q = static_cast<const BiCGScalars*>(g->hcsc->ptr);
    if (q->done != RUNNING || launched >= g->prm.coarse_maxiter) {
      g->coarse_iters += q->iter;
      g->coarse_solves += 1;
      g->last_coarse_iters = q->iter;
      if (eo)  // e_O = A_O^-1 r_O - (A^-1 H)_OE e_E, into the odd entries of the solution cv1
        coarse_stream(g, *g->Deo, 1, 1, 9, g->cv(1), g->cv(1), g->cv(8), MG_CR_NONE, nullptr, nullptr);
      return q->iter;
    }
  }
}

// ---- fine FP32 pieces of the cycle
// colour >= 0: only at the sites of that colour's blocks (the next SAP half
// sweep reads nothing else).
void fine_residual32(bridge_mg_s* g, const Field& b, const Field& x, const Field& out, int colour = -1) {
  // out = b - D x = b - T x + kappa H x
  for (int q = 0; q < 2; ++q) {
    HopCall c;
    c.prec = P_F32;
    c.flags = F_AUX | F_SELF | F_SELF_CLOV;
    c.red = R_NORM;
    c.cls = K_MG_RESID;
    c.out_parity = q;
    c.nrhs = 1;
    c.beta = g->op.kappa;
    c.s1 = -1.0;
    c.caux = 1.0;
    c.kcsw = op_kcsw(g->op);
    c.clov = g->clov.get();
    for (int k = 0; k < 4; ++k) c.bc[k] = g->op.bc[k];
    c.out = out.ptr(q);
    c.out_rs = out.rs;
    c.in = x.ptr(1 - q);
    c.in_rs = x.rs;
    c.self = x.ptr(q);
    c.self_rs = x.rs;
    c.aux = b.ptr(q);
    c.aux_rs = b.rs;
    if (colour >= 0) {
      c.site_map = reinterpret_cast<const uint32_t*>(g->smap->ptr) + g->soff[q][colour];
      c.n_map = (uint32_t)g->sn[q][colour];
      c.work_fraction = (double)g->sn[q][colour] / (double)g->L->vh;
    }
    run_hop(g->L, c, stream_of(g));
  }
}

// Raise the dynamic shared memory limit of a SAP kernel variant (once per
// device and size; at most 256 sites x 672 bytes = 168 KB).
template <bool CS>
void allow_sap_smem(long smem) {
  static std::mutex mu;
  static std::map<int, long> done;
  int dev = 0;
  BR_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lock(mu);
  if (done[dev] >= smem) return;
  BR_CUDA(cudaFuncSetAttribute(mg_sap_kernel<CS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  done[dev] = smem;
}

// fused: r is the right-hand side b and each block forms b - D x itself;
// otherwise r is the residual at the colour's sites.
void sap_half_sweep(bridge_mg_s* g, const Field& r, const Field& x, int colour, bool fused = false) {
  MgSapArgs a;
  std::memset(static_cast<void*>(&a), 0, sizeof(a));
  a.m = g->m;
  a.colour = colour;
  a.steps = g->prm.mr_steps;
  a.kappa = (float)g->op.kappa;
  a.fused = fused ? 1 : 0;
  for (int k = 0; k < 4; ++k) a.bcf[k] = (float)g->op.bc[k];
  a.r = r.ptr(0);
  a.x = x.ptr(0);
  a.field_block = r.block;
  a.gauge = gauge_ptr(g->L, P_F32);
  a.clov = clover_ptr(g->L, *g->clov, P_F32, false);
  const bool cs = g->sap_clover_smem != 0;
  const long smem = mg_sap_smem(g->m.bsites, cs);
  if (cs)
    allow_sap_smem<true>(smem);
  else
    allow_sap_smem<false>(smem);
  const double sites = (double)g->L->V / 2;
  // r, x in and out, the clover term, and the forward links of the hops that stay in the block
  double inner = 0;
  for (int k = 0; k < 4; ++k) inner += (double)(g->m.b[k] - 1) / g->m.b[k];
  double bytes = sites * (96 + 2 * 96 + 288 + 48 * inner);
  double flops = sites * g->prm.mr_steps * 1900.0;
  if (fused) {
    // the residual adds the forward links the block's own hops skip, the backward links across the
    // block faces and x at the neighbours in the other colour's blocks
    double faces = 0;
    for (int k = 0; k < 4; ++k) faces += 1.0 / g->m.b[k];
    bytes += sites * (48 * (4 - inner) + 48 * faces + 96 * 2 * faces);
    flops += sites * hop_cost(P_F32, F_AUX | F_SELF | F_SELF_CLOV, R_NONE).rhs_flops;
  }
  note_launch(g->L, K_MG_SAP, bytes, flops, stream_of(g), true);
  if (cs)
    mg_sap_kernel<true><<<g->m.nblocks / 2, block_threads(g), (size_t)smem, stream_of(g)>>>(a);
  else
    mg_sap_kernel<false><<<g->m.nblocks / 2, block_threads(g), (size_t)smem, stream_of(g)>>>(a);
  note_launch(g->L, K_MG_SAP, bytes, 0, stream_of(g), false);
  BR_CUDA(cudaGetLastError());
}

// Time both SAP kernel variants on a scratch residual (three half sweeps
// each, after one untimed) and keep the faster.  BRIDGE_MG_SAP=0 or 1 in the
// environment fixes the variant instead (1: clover term staged).
void pick_sap_variant(bridge_mg_s* g) {
  if (const char* e = std::getenv("BRIDGE_MG_SAP")) {
    if (e[0] == '0' || e[0] == '1') {
      g->sap_clover_smem = e[0] - '0';
      return;
    }
  }
  cudaStream_t st = stream_of(g);
  fill_scratch(g->r32, 7, st);
  BR_CUDA(cudaMemsetAsync(g->x32.buf->ptr, 0, g->x32.buf->bytes, st));
  cudaEvent_t e0, e1;
  BR_CUDA(cudaEventCreate(&e0));
  BR_CUDA(cudaEventCreate(&e1));
  float best = 0.f;
  int pick = 1;
  for (int v = 1; v >= 0; --v) {
    g->sap_clover_smem = v;
    sap_half_sweep(g, g->r32, g->x32, 0);
    BR_CUDA(cudaEventRecord(e0, st));
    for (int k = 0; k < 3; ++k) sap_half_sweep(g, g->r32, g->x32, k & 1);
    BR_CUDA(cudaEventRecord(e1, st));
    BR_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    BR_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    if (v == 1 || ms < best) {
      best = ms;
      pick = v;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  g->sap_clover_smem = pick;
}

// x = approximate D^-1 r by `cycles` SAP cycles added to x (x holds a start).
void sap(bridge_mg_s* g, const Field& r, const Field& x, int cycles, bool x_zero) {
  for (int cyc = 0; cyc < cycles; ++cyc)
    for (int colour = 0; colour < 2; ++colour) {
      if (cyc == 0 && colour == 0 && x_zero) {
        sap_half_sweep(g, r, x, colour);  // residual = r while x = 0
      } else if (g->sap_fused) {
        sap_half_sweep(g, r, x, colour, true);
      } else {
        fine_residual32(g, r, x, g->res32, colour);
        sap_half_sweep(g, g->res32, x, colour);
      }
    }
}

// z = M r: coarse correction then SAP post-smoothing (FP32 fields).
void cycle(bridge_mg_s* g, const Field& r, const Field& z) {
  restrict_to(g, r, g->cv(0));
  coarse_solve(g, g->cv(0));
  prolong_to(g, g->cv(1), z, false);
  sap(g, r, z, g->prm.sap_cycles, false);
}

void check_block(const bridge_lattice_s* L, const bridge_mg_params& p) {
  long bs = 1;
  for (int k = 0; k < 4; ++k) {
    BR_CHECK(p.block[k] >= 1 && L->dims[k] % p.block[k] == 0, BRIDGE_EINVAL, "mg block extents must divide the lattice");
    BR_CHECK((L->dims[k] / p.block[k]) % 2 == 0, BRIDGE_EINVAL, "mg needs an even number of blocks per direction");
    bs *= p.block[k];
  }
  BR_CHECK(bs <= 256 && bs >= 2, BRIDGE_EINVAL, "mg blocks hold 2 .. 256 sites");
  BR_CHECK(p.nvec >= 1 && p.nvec <= 32, BRIDGE_EINVAL, "mg nvec must be in 1..32");
  BR_CHECK(p.sap_cycles >= 0 && p.mr_steps >= 0 && p.coarse_maxiter >= 0 && p.setup_steps >= 0, BRIDGE_EINVAL,
           "mg iteration counts");
}

}  // namespace
}  // namespace bridge

// ============================================================== C-ABI
namespace bridge {
int mg_setup(bridge_lattice_s* L, const bridge_op& op, const bridge_mg_params& prm, const double* null_host,
             bridge_mg_s** out);
}

int bridge::mg_setup(bridge_lattice_s* L, const bridge_op& op, const bridge_mg_params& prm, const double* null_host,
                     bridge_mg_s** out) {
  check_block(L, prm);
  auto g = std::make_unique<bridge_mg_s>();
  g->L = L;
  g->op = op;
  g->prm = prm;
  g->m.g = L->g;
  g->m.bsites = 1;
  g->m.nblocks = 1;
  for (int k = 0; k < 4; ++k) {
    g->m.b[k] = prm.block[k];
    g->m.cd[k] = L->dims[k] / prm.block[k];
    g->m.bsites *= prm.block[k];
    g->m.nblocks *= g->m.cd[k];
  }
  g->nv = prm.nvec;
  g->n2 = 2 * prm.nvec;
  g->nc = (long)g->m.nblocks * g->n2;
  cudaStream_t st = L->stream;
  g->clov = clover_set(L, op_kcsw(op));
  gauge_ptr(L, P_F32);
  clover_ptr(L, *g->clov, P_F32, false);
  g->V = make_field(P_F32, BRIDGE_FULL, g->nv, L->vh);
  g->r32 = make_field(P_F32, BRIDGE_FULL, 1, L->vh);
  g->x32 = make_field(P_F32, BRIDGE_FULL, 1, L->vh);
  g->res32 = make_field(P_F32, BRIDGE_FULL, 1, L->vh);
  g->Dc.reset(new DevBuf((size_t)g->m.nblocks * 9 * g->n2 * g->n2 * sizeof(float2)));
  {
    std::vector<int> nb((size_t)g->m.nblocks * 9);
    for (int X = 0; X < g->m.nblocks; ++X)
      for (int d = 0; d < 9; ++d)
        nb[(size_t)X * 9 + d] = d == 0 ? X : mg_block_nbr(g->m, X, (d - 1) >> 1, ((d - 1) & 1) ? -1 : 1);
    g->cnbr.reset(new DevBuf(nb.size() * sizeof(int)));
    BR_CUDA(cudaMemcpy(g->cnbr->ptr, nb.data(), nb.size() * sizeof(int), cudaMemcpyHostToDevice));
  }
  g->cvec.reset(new DevBuf((size_t)11 * g->nc * sizeof(float2)));
  g->partial.reset(new DevBuf(sizeof(double2) * 1024 * 8));
  g->hpart.reset(new PinnedBuf(sizeof(double2) * 1024 * 8));
  g->csc.reset(new DevBuf(256));
  g->hcsc.reset(new PinnedBuf(256));
  BR_CUDA(cudaMemsetAsync(g->csc->ptr, 0, 256, st));
  g->cpart.reset(new DevBuf(sizeof(double) * 4 * std::max((g->nc + 255) / 256, coarse_tma_max_grid())));
  g->ccount.reset(new DevBuf(256));
  BR_CUDA(cudaMemsetAsync(g->ccount->ptr, 0, 256, st));
  // ---- the sites of each parity and block colour (for the SAP residuals)
  {
    std::vector<uint32_t> lists[2][2];
    const int* Ld = L->dims;
    const uint32_t lxh = (uint32_t)Ld[0] / 2;
    for (int p = 0; p < 2; ++p)
      for (int t = 0; t < Ld[3]; ++t)
        for (int z = 0; z < Ld[2]; ++z)
          for (int y = 0; y < Ld[1]; ++y)
            for (uint32_t xh = 0; xh < lxh; ++xh) {
              const int x = 2 * (int)xh + ((p + y + z + t) & 1);
              const int col = (x / g->m.b[0] + y / g->m.b[1] + z / g->m.b[2] + t / g->m.b[3]) & 1;
              const uint32_t ih = xh + lxh * (uint32_t)(y + Ld[1] * (z + Ld[2] * t));
              lists[p][col].push_back(ih);
            }
    std::vector<uint32_t> all;
    for (int p = 0; p < 2; ++p)
      for (int c = 0; c < 2; ++c) {
        g->soff[p][c] = (long)all.size();
        g->sn[p][c] = (long)lists[p][c].size();
        all.insert(all.end(), lists[p][c].begin(), lists[p][c].end());
      }
    g->smap.reset(new DevBuf(sizeof(uint32_t) * all.size()));
    BR_CUDA(cudaMemcpy(g->smap->ptr, all.data(), sizeof(uint32_t) * all.size(), cudaMemcpyHostToDevice));
  }
  const size_t canon = (size_t)L->V * 24;
  // ---- null vectors
  {
    DevBuf can(canon * g->nv * sizeof(double));
    if (null_host) {
      BR_CUDA(cudaMemcpyAsync(can.ptr, null_host, can.bytes, cudaMemcpyHostToDevice, st));
    } else {
      DevBuf eta(canon * sizeof(double));
      bridge_solver s;
      bridge_solver_defaults(&s);
      s.tol = prm.setup_tol;
      s.max_outer = 1;
      s.inner_tol = prm.setup_tol;
      for (int i = 0; i < g->nv; ++i) {
        note_launch(L, K_MG_SETUP, 0, 0, st, true);
        k_mg_random<<<grid_for((long)canon), 256, 0, st>>>(reinterpret_cast<double*>(eta.ptr), (long)canon, 1000u + i);
        note_launch(L, K_MG_SETUP, 0, 0, st, false);
        double* xi = reinterpret_cast<double*>(can.ptr) + canon * i;
        for (int step = 0; step < std::max(1, prm.setup_steps); ++step) {
          if (step > 0) {  // the next source is the last iterate (the scale does not matter)
            BR_CUDA(cudaMemcpyAsync(eta.ptr, xi, canon * sizeof(double), cudaMemcpyDeviceToDevice, st));
          }
          BR_CUDA(cudaMemsetAsync(xi, 0, canon * sizeof(double), st));
          SolveState S(L, op, s, 1, st, reinterpret_cast<double*>(eta.ptr), xi);
          while (!S.advance()) BR_CUDA(cudaEventSynchronize(S.wait_event()));
        }
      }
    }
    canon_to_field(L, reinterpret_cast<const double*>(can.ptr), g->V, st);
    BR_CUDA(cudaStreamSynchronize(st));
  }
  // ---- orthonormal aggregate bases
  {
    MgTransferArgs a = transfer_args(g.get());
    note_launch(L, K_MG_SETUP, 0, 0, st, true);
    mg_orthonormalize_kernel<<<g->m.nblocks, block_threads(g.get()), 0, st>>>(a);
    note_launch(L, K_MG_SETUP, 0, 0, st, false);
    BR_CUDA(cudaGetLastError());
  }
  // ---- coarse operator: probes of every basis column
  {
    Field w = make_field(P_F32, BRIDGE_FULL, 1, L->vh), y = make_field(P_F32, BRIDGE_FULL, 1, L->vh);
    MgProbeArgs pa;
    std::memset(static_cast<void*>(&pa), 0, sizeof(pa));
    pa.m = g->m;
    pa.kappa = (float)op.kappa;
    for (int k = 0; k < 4; ++k) pa.bcf[k] = (float)op.bc[k];
    pa.w = w.ptr(0);
    pa.y = y.ptr(0);
    pa.field_block = w.block;
    pa.gauge = gauge_ptr(L, P_F32);
    pa.clov = clover_ptr(L, *g->clov, P_F32, false);
    float2* tmp = g->cv(0);
    const long per_chi = 3L * L->vh;  // float4 plane-sites of one chirality in a parity block
    for (int chi = 0; chi < 2; ++chi)
      for (int i = 0; i < g->nv; ++i) {
        const int col = chi * g->nv + i;
        for (int p = 0; p < 2; ++p) {
          note_launch(L, K_MG_SETUP, 0, 0, st, true);
          k_mg_chiral<<<grid_for(6L * L->vh), 256, 0, st>>>(
              reinterpret_cast<const float4*>(g->V.buf->ptr + i * g->V.rs + p * g->V.block),
              reinterpret_cast<float4*>(w.ptr(p)), 6L * L->vh, per_chi, chi);
          note_launch(L, K_MG_SETUP, 0, 0, st, false);
        }
        for (int mode = 0; mode < 9; ++mode) {
          pa.mode = mode;
          note_launch(L, K_MG_SETUP, 0, 0, st, true);
          mg_probe_kernel<<<g->m.nblocks, block_threads(g.get()), 0, st>>>(pa);
          note_launch(L, K_MG_SETUP, 0, 0, st, false);
          restrict_to(g.get(), y, tmp);
          note_launch(L, K_MG_SETUP, 0, 0, st, true);
          k_mg_scatter_column<<<(unsigned)((g->nc + 255) / 256), 256, 0, st>>>(
              tmp, reinterpret_cast<float2*>(g->Dc->ptr), g->m.nblocks, g->n2, mode, col);
          note_launch(L, K_MG_SETUP, 0, 0, st, false);
        }
      }
    BR_CUDA(cudaGetLastError());
    if (prm.coarse_half) {
      const long n = (long)g->m.nblocks * 9 * g->n2 * g->n2;
      g->Dch.reset(new DevBuf(sizeof(__half2) * n));
      note_launch(L, K_MG_SETUP, 0, 0, st, true);
      k_mg_to_half<<<grid_for(n), 256, 0, st>>>(reinterpret_cast<const float2*>(g->Dc->ptr),
                                                   reinterpret_cast<__half2*>(g->Dch->ptr), (long)g->m.nblocks * 9,
                                                   g->n2, mg_coarse_unrolled(g->n2) ? 1 : 0);
      note_launch(L, K_MG_SETUP, 0, 0, st, false);
      BR_CUDA(cudaGetLastError());
      if (prm.coarse_eo && mg_coarse_unrolled(g->n2)) {
        // the even-odd tiles: A_X^-1 and A_X^-1 times the hopping couplings, then FP16 tiled
        const int n2 = g->n2;
        DevBuf ainv(sizeof(float2) * (size_t)g->m.nblocks * n2 * n2), deo(sizeof(float2) * (size_t)n);
        const size_t inv_smem = sizeof(float2) * (size_t)(2 * n2 * n2 + n2);
        DevBuf singular(sizeof(int));
        BR_CUDA(cudaMemsetAsync(singular.ptr, 0, sizeof(int), st));
        note_launch(L, K_MG_SETUP, 0, 0, st, true);
        mg_invert_self_kernel<<<g->m.nblocks, 256, inv_smem, st>>>(reinterpret_cast<const float2*>(g->Dc->ptr),
                                                                   reinterpret_cast<float2*>(ainv.ptr), n2,
                                                                   reinterpret_cast<int*>(singular.ptr));
        mg_premul_kernel<<<g->m.nblocks, 256, sizeof(float2) * (size_t)n2 * n2, st>>>(
            reinterpret_cast<const float2*>(g->Dc->ptr), reinterpret_cast<const float2*>(ainv.ptr),
            reinterpret_cast<float2*>(deo.ptr), n2);
        g->Deo.reset(new DevBuf(sizeof(__half2) * n));
        k_mg_to_half<<<grid_for(n), 256, 0, st>>>(reinterpret_cast<const float2*>(deo.ptr),
                                                     reinterpret_cast<__half2*>(g->Deo->ptr), (long)g->m.nblocks * 9,
                                                     n2, 1);
        note_launch(L, K_MG_SETUP, 0, 0, st, false);
        BR_CUDA(cudaGetLastError());
        int sing = 0;
        BR_CUDA(cudaMemcpyAsync(&sing, singular.ptr, sizeof(int), cudaMemcpyDeviceToHost, st));
        BR_CUDA(cudaStreamSynchronize(st));  // the temporaries are freed on return
        if (sing) g->Deo.reset();  // a numerically singular self coupling: solve the full coarse system
      }
    }
    BR_CUDA(cudaStreamSynchronize(st));
  }
  pick_sap_variant(g.get());
  if (const char* e = std::getenv("BRIDGE_MG_SAP_FUSED")) g->sap_fused = e[0] != '0';
  *out = g.release();
  return BRIDGE_OK;
}

namespace bridge {

// Flat vector operations on full fields of one precision (T = float2 for
// FP32, double2 for FP64): each parity block holds 12 vh complex numbers.
template <class T>
void gaxpy(bridge_mg_s* g, cx<double> a, const Field& x, cx<double> b, const Field& y, cx<double> c, const Field* z) {
  for (int p = 0; p < 2; ++p)
    vaxpy<T>(g, fine_n(x), a, reinterpret_cast<const T*>(x.ptr(p)), b, reinterpret_cast<T*>(y.ptr(p)), c,
             z ? reinterpret_cast<const T*>(z->ptr(p)) : nullptr);
}
template <class T>
std::vector<cx<double>> gdots(bridge_mg_s* g, std::initializer_list<std::pair<const Field*, const Field*>> pairs) {
  int slot = 0;
  for (const auto& pr : pairs)
    for (int p = 0; p < 2; ++p)
      vdot_launch<T>(g, fine_n(*pr.first), reinterpret_cast<const T*>(pr.first->ptr(p)),
                     reinterpret_cast<const T*>(pr.second->ptr(p)), slot++);
  auto parts = vdot_collect(g, slot);
  std::vector<cx<double>> out;
  for (size_t k = 0; k < parts.size(); k += 2) out.push_back(parts[k] + parts[k + 1]);
  return out;
}

// FBiCGStab in FP32 on D e = r (e = 0 on entry), preconditioned by the cycle,
// to ||r - D e|| <= tol ||r|| by the recursive residual; returns iterations.
int fbicgstab32(bridge_mg_s* g, const Field& rhs, const Field& x, double tol, int max_iter, int& restarts) {
  bridge_lattice_s* L = g->L;
  cudaStream_t st = L->stream;
  auto F = [&](const char* name) -> Field& { return workspace(L, std::string("mg_") + name, P_F32, BRIDGE_FULL, 1); };
  Field &r = F("r"), &rh = F("rh"), &p = F("p"), &v = F("v"), &sv = F("s"), &t = F("t"), &ph = F("ph"), &sh = F("sh");
  auto Dop = [&](const Field& in, const Field& out) { apply_d(L, g->op, out, in, st); };
  const cx<double> one{1, 0}, zero{0, 0};
  BR_CUDA(cudaMemsetAsync(x.buf->ptr, 0, x.buf->bytes, st));
  BR_CUDA(cudaMemcpyAsync(r.buf->ptr, rhs.buf->ptr, r.buf->bytes, cudaMemcpyDeviceToDevice, st));
  const double b2 = gdots<float2>(g, {{&r, &r}})[0].r;
  if (!(b2 > 0.0)) return 0;
  const double tol2 = tol * tol * b2;
  double r2 = b2;
  int it = 0;
  while (it < max_iter && r2 > tol2) {
    BR_CUDA(cudaMemcpyAsync(rh.buf->ptr, r.buf->ptr, r.buf->bytes, cudaMemcpyDeviceToDevice, st));
    BR_CUDA(cudaMemsetAsync(p.buf->ptr, 0, p.buf->bytes, st));
    BR_CUDA(cudaMemsetAsync(v.buf->ptr, 0, v.buf->bytes, st));
    cx<double> rho{1, 0}, alpha{1, 0}, omega{1, 0};
    bool breakdown = false;
    while (it < max_iter && r2 > tol2) {
      const cx<double> rho_new = gdots<float2>(g, {{&rh, &r}})[0];
      if (std::hypot(rho_new.r, rho_new.i) < 1e-30 * std::sqrt(r2 * b2)) {
        breakdown = true;
        break;
      }
      const cx<double> beta = (rho_new * cx<double>{1.0 / (rho.r * rho.r + rho.i * rho.i), 0} * conj(rho)) *
                              (alpha * cx<double>{1.0 / (omega.r * omega.r + omega.i * omega.i), 0} * conj(omega));
      gaxpy<float2>(g, one, r, beta, p, cx<double>{0, 0} - beta * omega, &v);  // p = r + beta (p - omega v)
      cycle(g, p, ph);
      Dop(ph, v);
      const cx<double> rv = gdots<float2>(g, {{&rh, &v}})[0];
      const double rv2 = rv.r * rv.r + rv.i * rv.i;
      if (!(rv2 > 0.0)) {
        breakdown = true;
        break;
      }
      alpha = rho_new * cx<double>{1.0 / rv2, 0} * conj(rv);
      gaxpy<float2>(g, one, r, zero, sv, cx<double>{0, 0} - alpha, &v);  // s = r - alpha v
      cycle(g, sv, sh);
      Dop(sh, t);
      auto d = gdots<float2>(g, {{&t, &sv}, {&t, &t}});
      omega = d[1].r > 0 ? d[0] * cx<double>{1.0 / d[1].r, 0} : zero;
      gaxpy<float2>(g, alpha, ph, one, x, omega, &sh);                   // x += alpha p^ + omega s^
      gaxpy<float2>(g, one, sv, zero, r, cx<double>{0, 0} - omega, &t);  // r = s - omega t
      r2 = gdots<float2>(g, {{&r, &r}})[0].r;
      rho = rho_new;
      ++it;
      if (omega.r == 0.0 && omega.i == 0.0) {
        breakdown = true;
        break;
      }
    }
    if (!breakdown) break;
    restarts += 1;  // restart from the recursive residual with a fresh shadow vector
  }
  return it;
}

// D x = b in FP64 by defect correction: r = b - D x (FP64), an FP32
// FBiCGStab pass with the multigrid cycle on D e = r, x += e; b, x
// canonical FP64 on the device (x: guess in, solution out).
void mg_solve_one(bridge_mg_s* g, const double* b_dev, double* x_dev, const bridge_solver& s, bridge_info& info) {
  bridge_lattice_s* L = g->L;
  cudaStream_t st = L->stream;
  const auto t0 = std::chrono::steady_clock::now();
  Field& b = workspace(L, "mg_b64", P_F64, BRIDGE_FULL, 1);
  Field& x = workspace(L, "mg_x64", P_F64, BRIDGE_FULL, 1);
  Field& r = workspace(L, "mg_r64", P_F64, BRIDGE_FULL, 1);
  Field& r32 = workspace(L, "mg_rin", P_F32, BRIDGE_FULL, 1);
  Field& e32 = workspace(L, "mg_e", P_F32, BRIDGE_FULL, 1);
  canon_to_field(L, b_dev, b, st);
  canon_to_field(L, x_dev, x, st);
  std::memset(&info, 0, sizeof(info));
  const cx<double> one{1, 0}, zero{0, 0};
  const double b2 = gdots<double2>(g, {{&b, &b}})[0].r;
  if (!(b2 > 0.0)) {
    BR_CUDA(cudaMemsetAsync(x.buf->ptr, 0, x.buf->bytes, st));
    field_to_canon(L, x, x_dev, st);
    BR_CUDA(cudaStreamSynchronize(st));
    info.status = BRIDGE_OK;
    return;
  }
  const double floor_tol = s.inner_tol > 0 ? s.inner_tol : 1e-6;
  const int max_iter = s.max_iter > 0 ? s.max_iter : 1000;
  const int max_outer = s.max_outer > 0 ? s.max_outer : 50;
  int status = BRIDGE_ENOCONV;
  double r2_prev = 0.0, tau = floor_tol;
  for (int pass = 0;; ++pass) {
    apply_d(L, g->op, r, x, st);
    gaxpy<double2>(g, one, b, cx<double>{-1, 0}, r, zero, nullptr);  // r = b - D x
    const double r2 = gdots<double2>(g, {{&r, &r}})[0].r;
    info.true_rel_residual = std::sqrt(r2 / b2);
    info.outer_iters = pass;
    if (r2 <= s.tol * s.tol * b2) {
      status = BRIDGE_OK;
      break;
    }
    if (!std::isfinite(r2)) {
      status = BRIDGE_EBREAKDOWN;
      break;
    }
    if (pass >= max_outer || info.inner_iters >= max_iter) break;
    tau = next_inner_tol(floor_tol, s.tol, b2, r2, r2_prev, tau, pass == 0);
    r2_prev = r2;
    convert_field(L, r, r32, 0, st, nullptr);
    convert_field(L, r, r32, 1, st, nullptr);
    info.inner_iters += fbicgstab32(g, r32, e32, tau, max_iter - info.inner_iters, info.restarts);
    accumulate64(L, e32, 0, x, 0, st, nullptr);
    accumulate64(L, e32, 1, x, 1, st, nullptr);
  }
  field_to_canon(L, x, x_dev, st);
  BR_CUDA(cudaStreamSynchronize(st));
  info.status = status;
  info.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

// Diagnostic applications on canonical FP64 device buffers.
void mg_apply(bridge_mg_s* g, int which, const double* in, double* out) {
  bridge_lattice_s* L = g->L;
  cudaStream_t st = L->stream;
  const long nc = g->nc;
  DevBuf cin(sizeof(float2) * nc), cout(sizeof(float2) * nc);
  auto c64_to_32 = [&](const double* src, float2* dst) {
    std::vector<double> h(2 * nc);
    BR_CUDA(cudaMemcpy(h.data(), src, sizeof(double) * 2 * nc, cudaMemcpyDeviceToHost));
    std::vector<float2> f(nc);
    for (long k = 0; k < nc; ++k) f[k] = make_float2((float)h[2 * k], (float)h[2 * k + 1]);
    BR_CUDA(cudaMemcpy(dst, f.data(), sizeof(float2) * nc, cudaMemcpyHostToDevice));
  };
  auto c32_to_64 = [&](const float2* src, double* dst) {
    std::vector<float2> f(nc);
    BR_CUDA(cudaStreamSynchronize(st));
    BR_CUDA(cudaMemcpy(f.data(), src, sizeof(float2) * nc, cudaMemcpyDeviceToHost));
    std::vector<double> h(2 * nc);
    for (long k = 0; k < nc; ++k) {
      h[2 * k] = f[k].x;
      h[2 * k + 1] = f[k].y;
    }
    BR_CUDA(cudaMemcpy(dst, h.data(), sizeof(double) * 2 * nc, cudaMemcpyHostToDevice));
  };
  switch (which) {
    case BRIDGE_MG_RESTRICT:
      canon_to_field(L, in, g->r32, st);
      restrict_to(g, g->r32, reinterpret_cast<float2*>(cout.ptr));
      c32_to_64(reinterpret_cast<float2*>(cout.ptr), out);
      break;
    case BRIDGE_MG_PROLONG:
      c64_to_32(in, reinterpret_cast<float2*>(cin.ptr));
      prolong_to(g, reinterpret_cast<float2*>(cin.ptr), g->x32, false);
      field_to_canon(L, g->x32, out, st);
      break;
    case BRIDGE_MG_COARSE:
      c64_to_32(in, reinterpret_cast<float2*>(cin.ptr));
      coarse_apply(g, reinterpret_cast<float2*>(cin.ptr), reinterpret_cast<float2*>(cout.ptr));
      c32_to_64(reinterpret_cast<float2*>(cout.ptr), out);
      break;
    case BRIDGE_MG_COARSE_HALF:
      if (!g->Dch) throw Error{BRIDGE_EINVAL, "no FP16 coarse operator (coarse_half = 0)"};
      clear_coarse_err(g);
      c64_to_32(in, reinterpret_cast<float2*>(cin.ptr));
      coarse_apply(g, reinterpret_cast<float2*>(cin.ptr), reinterpret_cast<float2*>(cout.ptr), nullptr, MG_CR_NONE,
                   nullptr, true);
      c32_to_64(reinterpret_cast<float2*>(cout.ptr), out);
      BR_CUDA(cudaMemcpy(g->hcsc->ptr, g->csc->ptr, 256, cudaMemcpyDeviceToHost));
      check_coarse_err(g);
      break;
    case BRIDGE_MG_COARSE_SOLVE:
      c64_to_32(in, reinterpret_cast<float2*>(cin.ptr));
      coarse_solve(g, reinterpret_cast<float2*>(cin.ptr));
      c32_to_64(g->cv(1), out);
      break;
    case BRIDGE_MG_SAP:
      canon_to_field(L, in, g->r32, st);
      BR_CUDA(cudaMemsetAsync(g->x32.buf->ptr, 0, g->x32.buf->bytes, st));
      sap(g, g->r32, g->x32, g->prm.sap_cycles, true);
      field_to_canon(L, g->x32, out, st);
      break;
    case BRIDGE_MG_CYCLE:
      canon_to_field(L, in, g->r32, st);
      cycle(g, g->r32, g->x32);
      field_to_canon(L, g->x32, out, st);
      break;
    default:
      throw Error{BRIDGE_EINVAL, "unknown multigrid application"};
  }
  BR_CUDA(cudaStreamSynchronize(st));
}

}  // namespace bridge

#define BR_MG_BEGIN try {
#define BR_MG_END                              \
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

extern "C" {

void bridge_mg_defaults(bridge_mg_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  for (int k = 0; k < 4; ++k) p->block[k] = 4;
  p->nvec = 16;
  p->setup_tol = 5e-2;
  p->setup_steps = 1;
  p->sap_cycles = 2;
  p->mr_steps = 4;
  p->coarse_tol = 5e-2;
  p->coarse_maxiter = 200;
  p->coarse_half = 1;
  p->coarse_eo = 1;
}

int bridge_mg_setup(bridge_lattice L, const bridge_op* op, const bridge_mg_params* prm, const double* null_vectors,
                    bridge_mg* out) {
  BR_MG_BEGIN
  BR_CHECK(L && op && prm && out, BRIDGE_EINVAL, "NULL argument");
  BR_CHECK(L->have_gauge, BRIDGE_ESTATE, "no gauge field uploaded");
  BR_CHECK(op->kind == BRIDGE_WILSON || op->kind == BRIDGE_CLOVER, BRIDGE_EINVAL,
           "multigrid takes WILSON and CLOVER operators");
  for (int k = 0; k < 4; ++k) BR_CHECK(op->bc[k] == 1 || op->bc[k] == -1, BRIDGE_EINVAL, "op.bc must be +1 or -1");
  *out = nullptr;
  std::lock_guard<std::mutex> lk(L->api_mu);
  bridge_mg_s* g = nullptr;
  mg_setup(L, *op, *prm, null_vectors, &g);
  *out = g;
  BR_MG_END
}

int bridge_mg_destroy(bridge_mg g) {
  BR_MG_BEGIN
  if (!g) return BRIDGE_OK;
  cudaStreamSynchronize(g->L->stream);
  delete g;
  BR_MG_END
}

int bridge_mg_solve(bridge_mg g, const bridge_solver* s, const double* b, double* x, int nrhs, bridge_info* info) {
  BR_MG_BEGIN
  BR_CHECK(g && s && b && x, BRIDGE_EINVAL, "NULL argument");
  BR_CHECK(s->tol > 0 && std::isfinite(s->tol), BRIDGE_EINVAL, "tol must be > 0");
  BR_CHECK(nrhs >= 0, BRIDGE_EINVAL, "nrhs < 0");
  bridge_lattice_s* L = g->L;
  std::lock_guard<std::mutex> lk(L->api_mu);
  const size_t n = (size_t)L->V * 24;
  DevBuf db(n * sizeof(double)), dx(n * sizeof(double));
  int status = BRIDGE_OK;
  for (int r = 0; r < nrhs; ++r) {
    BR_CUDA(cudaMemcpyAsync(db.ptr, b + n * r, n * sizeof(double), cudaMemcpyHostToDevice, L->stream));
    BR_CUDA(cudaMemcpyAsync(dx.ptr, x + n * r, n * sizeof(double), cudaMemcpyHostToDevice, L->stream));
    bridge_info inf;
    mg_solve_one(g, reinterpret_cast<double*>(db.ptr), reinterpret_cast<double*>(dx.ptr), *s, inf);
    BR_CUDA(cudaMemcpy(x + n * r, dx.ptr, n * sizeof(double), cudaMemcpyDeviceToHost));
    if (info) info[r] = inf;
    if (inf.status != BRIDGE_OK) status = inf.status;
  }
  if (status != BRIDGE_OK) set_error(status, "multigrid solve did not reach tolerance");
  return status;
  BR_MG_END
}

int bridge_mg_solve_dev(bridge_mg g, const bridge_solver* s, const double* b, double* x, int nrhs, bridge_info* info) {
  BR_MG_BEGIN
  BR_CHECK(g && s && b && x, BRIDGE_EINVAL, "NULL argument");
  BR_CHECK(s->tol > 0 && std::isfinite(s->tol), BRIDGE_EINVAL, "tol must be > 0");
  BR_CHECK(nrhs >= 0, BRIDGE_EINVAL, "nrhs < 0");
  bridge_lattice_s* L = g->L;
  std::lock_guard<std::mutex> lk(L->api_mu);
  const size_t n = (size_t)L->V * 24;
  int status = BRIDGE_OK;
  for (int r = 0; r < nrhs; ++r) {
    bridge_info inf;
    mg_solve_one(g, b + n * r, x + n * r, *s, inf);
    if (info) info[r] = inf;
    if (inf.status != BRIDGE_OK) status = inf.status;
  }
  if (status != BRIDGE_OK) set_error(status, "multigrid solve did not reach tolerance");
  return status;
  BR_MG_END
}

int bridge_mg_apply(bridge_mg g, int which, const double* in, double* out) {
  BR_MG_BEGIN
  BR_CHECK(g && in && out, BRIDGE_EINVAL, "NULL argument");
  bridge_lattice_s* L = g->L;
  std::lock_guard<std::mutex> lk(L->api_mu);
  const bool fine_in = which == BRIDGE_MG_RESTRICT || which == BRIDGE_MG_SAP || which == BRIDGE_MG_CYCLE;
  const bool fine_out = which == BRIDGE_MG_PROLONG || which == BRIDGE_MG_SAP || which == BRIDGE_MG_CYCLE;
  const size_t nf = (size_t)L->V * 24, ncd = (size_t)g->nc * 2;
  const size_t nin = fine_in ? nf : ncd, nout = fine_out ? nf : ncd;
  DevBuf din(nin * sizeof(double)), dout(nout * sizeof(double));
  BR_CUDA(cudaMemcpy(din.ptr, in, nin * sizeof(double), cudaMemcpyHostToDevice));
  mg_apply(g, which, reinterpret_cast<double*>(din.ptr), reinterpret_cast<double*>(dout.ptr));
  BR_CUDA(cudaMemcpy(out, dout.ptr, nout * sizeof(double), cudaMemcpyDeviceToHost));
  BR_MG_END
}

int bridge_mg_coarse_matrix(bridge_mg g, double* out) {
  BR_MG_BEGIN
  BR_CHECK(g && out, BRIDGE_EINVAL, "NULL argument");
  const size_t n = (size_t)g->m.nblocks * 9 * g->n2 * g->n2;
  std::vector<float2> h(n);
  BR_CUDA(cudaStreamSynchronize(g->L->stream));
  BR_CUDA(cudaMemcpy(h.data(), g->Dc->ptr, n * sizeof(float2), cudaMemcpyDeviceToHost));
  for (size_t k = 0; k < n; ++k) {
    out[2 * k] = h[k].x;
    out[2 * k + 1] = h[k].y;
  }
  BR_MG_END
}

int bridge_mg_counters(bridge_mg g, long* coarse_solves, long* coarse_iters) {
  if (!g) return BRIDGE_EINVAL;
  if (coarse_solves) *coarse_solves = g->coarse_solves;
  if (coarse_iters) *coarse_iters = g->coarse_iters;
  return BRIDGE_OK;
}

int bridge_mg_info(bridge_mg g, int* nblocks, int* nvec) {
  if (!g) return BRIDGE_EINVAL;
  if (nblocks) *nblocks = g->m.nblocks;
  if (nvec) *nvec = g->nv;
  return BRIDGE_OK;
}

}  // extern "C"
