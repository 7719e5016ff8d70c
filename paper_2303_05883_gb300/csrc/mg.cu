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
//   solve   FBiCGStab in FP64 on D with the cycle as the preconditioner.
// The scalars of the coarse BiCGStab and of the outer solver live on the
// host: each of their iterations costs one preconditioner cycle or one coarse
// operator application, far more than the reads of the scalars.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
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
  std::unique_ptr<DevBuf> Dc, cvec, partial;
  std::unique_ptr<PinnedBuf> hpart;
  Field r32, x32, res32;  // fine FP32 work fields of the cycle
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
void faxpy(bridge_mg_s* g, cx<double> a, const Field& x, cx<double> b, const Field& y, cx<double> c, const Field* z) {
  for (int p = 0; p < 2; ++p)
    vaxpy<double2>(g, fine_n(x), a, reinterpret_cast<const double2*>(x.ptr(p)), b, reinterpret_cast<double2*>(y.ptr(p)),
                   c, z ? reinterpret_cast<const double2*>(z->ptr(p)) : nullptr);
}
// <x, y> for the listed pairs, computed together (one host wait)
std::vector<cx<double>> fdots(bridge_mg_s* g, std::initializer_list<std::pair<const Field*, const Field*>> pairs) {
  int slot = 0;
  for (const auto& pr : pairs)
    for (int p = 0; p < 2; ++p)
      vdot_launch<double2>(g, fine_n(*pr.first), reinterpret_cast<const double2*>(pr.first->ptr(p)),
                           reinterpret_cast<const double2*>(pr.second->ptr(p)), slot++);
  auto parts = vdot_collect(g, slot);
  std::vector<cx<double>> out;
  for (size_t k = 0; k < parts.size(); k += 2) out.push_back(parts[k] + parts[k + 1]);
  return out;
}

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
void coarse_apply(bridge_mg_s* g, const float2* x, float2* y, const float2* b = nullptr) {
  MgCoarseArgs a;
  a.m = g->m;
  a.n2 = g->n2;
  a.Dc = reinterpret_cast<const float2*>(g->Dc->ptr);
  a.x = x;
  a.b = b;
  a.y = y;
  const long n = g->nc;
  const double bytes = (double)g->m.nblocks * 9 * g->n2 * g->n2 * 8 + n * 8.0 * (b ? 3 : 2);
  note_launch(g->L, K_MG_COARSE, bytes, (double)g->m.nblocks * 9 * g->n2 * g->n2 * 8, stream_of(g), true);
  mg_coarse_kernel<<<(unsigned)((n + 255) / 256), 256, 0, stream_of(g)>>>(a);
  note_launch(g->L, K_MG_COARSE, bytes, 0, stream_of(g), false);
  BR_CUDA(cudaGetLastError());
}

// ---- coarse BiCGStab (host scalars): D_c e = r to a relative tolerance
int coarse_solve(bridge_mg_s* g, const float2* rhs, float2* x) {
  const long n = g->nc;
  float2 *r = g->cv(2), *rh = g->cv(3), *p = g->cv(4), *v = g->cv(5), *s = g->cv(6), *t = g->cv(7);
  const cx<double> one{1, 0}, zero{0, 0};
  BR_CUDA(cudaMemsetAsync(x, 0, sizeof(float2) * n, stream_of(g)));
  BR_CUDA(cudaMemcpyAsync(r, rhs, sizeof(float2) * n, cudaMemcpyDeviceToDevice, stream_of(g)));
  BR_CUDA(cudaMemcpyAsync(rh, rhs, sizeof(float2) * n, cudaMemcpyDeviceToDevice, stream_of(g)));
  BR_CUDA(cudaMemsetAsync(p, 0, sizeof(float2) * n, stream_of(g)));
  BR_CUDA(cudaMemsetAsync(v, 0, sizeof(float2) * n, stream_of(g)));
  vdot_launch<float2>(g, n, rhs, rhs, 0);
  const double b2 = vdot_collect(g, 1)[0].r;
  if (!(b2 > 0.0)) return 0;
  const double tol2 = g->prm.coarse_tol * g->prm.coarse_tol * b2;
  cx<double> rho{1, 0}, alpha{1, 0}, omega{1, 0};
  double r2 = b2;
  int it = 0;
  for (; it < g->prm.coarse_maxiter && r2 > tol2; ++it) {
    vdot_launch<float2>(g, n, rh, r, 0);
    const cx<double> rho_new = vdot_collect(g, 1)[0];
    if (std::hypot(rho_new.r, rho_new.i) == 0.0) break;
    const cx<double> beta = (rho_new * cx<double>{1.0 / (rho.r * rho.r + rho.i * rho.i), 0} * conj(rho)) *
                            (alpha * cx<double>{1.0 / (omega.r * omega.r + omega.i * omega.i), 0} * conj(omega));
    // p = r + beta (p - omega v)
    vaxpy<float2>(g, n, one, r, beta, p, cx<double>{0, 0} - beta * omega, v);
    coarse_apply(g, p, v);
    vdot_launch<float2>(g, n, rh, v, 0);
    const cx<double> rv = vdot_collect(g, 1)[0];
    const double rv2 = rv.r * rv.r + rv.i * rv.i;
    if (!(rv2 > 0.0)) break;
    alpha = rho_new * cx<double>{1.0 / rv2, 0} * conj(rv);
    vaxpy<float2>(g, n, one, r, zero, s, cx<double>{0, 0} - alpha, v);  // s = r - alpha v
    coarse_apply(g, s, t);
    vdot_launch<float2>(g, n, t, s, 0);
    vdot_launch<float2>(g, n, t, t, 1);
    auto d = vdot_collect(g, 2);
    omega = d[1].r > 0 ? d[0] * cx<double>{1.0 / d[1].r, 0} : zero;
    vaxpy<float2>(g, n, alpha, p, one, x, omega, s);                       // x += alpha p + omega s
    vaxpy<float2>(g, n, one, s, zero, r, cx<double>{0, 0} - omega, t);     // r = s - omega t
    vdot_launch<float2>(g, n, r, r, 0);
    r2 = vdot_collect(g, 1)[0].r;
    rho = rho_new;
    if (omega.r == 0.0 && omega.i == 0.0) break;
  }
  return it;
}

// ---- fine FP32 pieces of the cycle
void fine_residual32(bridge_mg_s* g, const Field& b, const Field& x, const Field& out) {
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
    run_hop(g->L, c, stream_of(g));
  }
}

void sap_half_sweep(bridge_mg_s* g, const Field& r, const Field& x, int colour) {
  MgSapArgs a;
  std::memset(static_cast<void*>(&a), 0, sizeof(a));
  a.m = g->m;
  a.colour = colour;
  a.steps = g->prm.mr_steps;
  a.kappa = (float)g->op.kappa;
  a.r = r.ptr(0);
  a.x = x.ptr(0);
  a.field_block = r.block;
  a.gauge = gauge_ptr(g->L, P_F32);
  a.clov = clover_ptr(g->L, *g->clov, P_F32, false);
  const long smem = 12L * g->m.bsites * 8;
  const double sites = (double)g->L->V / 2;
  const double bytes = sites * (96 + 2 * 96 + 8 * 48 + 288);
  note_launch(g->L, K_MG_SAP, bytes, sites * g->prm.mr_steps * 1900.0, stream_of(g), true);
  mg_sap_kernel<<<g->m.nblocks, block_threads(g), (size_t)smem, stream_of(g)>>>(a);
  note_launch(g->L, K_MG_SAP, bytes, 0, stream_of(g), false);
  BR_CUDA(cudaGetLastError());
}

// x = approximate D^-1 r by `cycles` SAP cycles added to x (x holds a start).
void sap(bridge_mg_s* g, const Field& r, const Field& x, int cycles, bool x_zero) {
  for (int cyc = 0; cyc < cycles; ++cyc)
    for (int colour = 0; colour < 2; ++colour) {
      if (cyc == 0 && colour == 0 && x_zero) {
        sap_half_sweep(g, r, x, colour);  // residual = r while x = 0
      } else {
        fine_residual32(g, r, x, g->res32);
        sap_half_sweep(g, g->res32, x, colour);
      }
    }
}

// z = M r: coarse correction then SAP post-smoothing (FP32 fields).
void cycle(bridge_mg_s* g, const Field& r, const Field& z) {
  restrict_to(g, r, g->cv(0));
  coarse_solve(g, g->cv(0), g->cv(1));
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
  BR_CHECK(p.sap_cycles >= 0 && p.mr_steps >= 0 && p.coarse_maxiter >= 0, BRIDGE_EINVAL, "mg iteration counts");
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
  g->cvec.reset(new DevBuf((size_t)8 * g->nc * sizeof(float2)));
  g->partial.reset(new DevBuf(sizeof(double2) * 1024 * 8));
  g->hpart.reset(new PinnedBuf(sizeof(double2) * 1024 * 8));
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
        BR_CUDA(cudaMemsetAsync(xi, 0, canon * sizeof(double), st));
        SolveState S(L, op, s, 1, st, reinterpret_cast<double*>(eta.ptr), xi);
        while (!S.advance()) BR_CUDA(cudaEventSynchronize(S.wait_event()));
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
    BR_CUDA(cudaStreamSynchronize(st));
  }
  *out = g.release();
  return BRIDGE_OK;
}

namespace bridge {

// FBiCGStab (FP64) on D x = b, preconditioned by the FP32 cycle; b, x
// canonical FP64 on the device (x: guess in, solution out).
void mg_solve_one(bridge_mg_s* g, const double* b_dev, double* x_dev, const bridge_solver& s, bridge_info& info) {
  bridge_lattice_s* L = g->L;
  cudaStream_t st = L->stream;
  const auto t0 = std::chrono::steady_clock::now();
  auto F = [&] { return make_field(P_F64, BRIDGE_FULL, 1, L->vh); };
  Field b = F(), x = F(), r = F(), rh = F(), p = F(), v = F(), sv = F(), t = F(), ph = F(), sh = F();
  canon_to_field(L, b_dev, b, st);
  canon_to_field(L, x_dev, x, st);
  std::memset(&info, 0, sizeof(info));
  auto Dop = [&](const Field& in, const Field& out) { apply_d(L, g->op, out, in, st); };
  auto prec = [&](const Field& in, const Field& out) {
    convert_field(L, in, g->r32, 0, st, nullptr);
    convert_field(L, in, g->r32, 1, st, nullptr);
    cycle(g, g->r32, g->x32);
    convert_field(L, g->x32, out, 0, st, nullptr);
    convert_field(L, g->x32, out, 1, st, nullptr);
  };
  const cx<double> one{1, 0}, zero{0, 0};
  const double b2 = fdots(g, {{&b, &b}})[0].r;
  if (!(b2 > 0.0)) {
    BR_CUDA(cudaMemsetAsync(x.buf->ptr, 0, x.buf->bytes, st));
    field_to_canon(L, x, x_dev, st);
    BR_CUDA(cudaStreamSynchronize(st));
    info.status = BRIDGE_OK;
    return;
  }
  const double tol2 = s.tol * s.tol * b2;
  const int max_iter = s.max_iter > 0 ? s.max_iter : 1000;
  int status = BRIDGE_ENOCONV;
  for (int restart = 0; restart < 10 && info.inner_iters < max_iter; ++restart) {
    // r = b - D x (true residual)
    Dop(x, t);
    faxpy(g, one, b, zero, r, cx<double>{-1, 0}, &t);
    double r2 = fdots(g, {{&r, &r}})[0].r;
    info.true_rel_residual = std::sqrt(r2 / b2);
    if (r2 <= tol2) {
      status = BRIDGE_OK;
      break;
    }
    info.outer_iters = restart;
    BR_CUDA(cudaMemcpyAsync(rh.buf->ptr, r.buf->ptr, r.buf->bytes, cudaMemcpyDeviceToDevice, st));
    BR_CUDA(cudaMemsetAsync(p.buf->ptr, 0, p.buf->bytes, st));
    BR_CUDA(cudaMemsetAsync(v.buf->ptr, 0, v.buf->bytes, st));
    cx<double> rho{1, 0}, alpha{1, 0}, omega{1, 0};
    bool breakdown = false;
    while (r2 > tol2 && info.inner_iters < max_iter) {
      const cx<double> rho_new = fdots(g, {{&rh, &r}})[0];
      if (std::hypot(rho_new.r, rho_new.i) < 1e-30 * std::sqrt(r2 * b2)) {
        breakdown = true;
        break;
      }
      const cx<double> beta = (rho_new * cx<double>{1.0 / (rho.r * rho.r + rho.i * rho.i), 0} * conj(rho)) *
                              (alpha * cx<double>{1.0 / (omega.r * omega.r + omega.i * omega.i), 0} * conj(omega));
      faxpy(g, one, r, beta, p, cx<double>{0, 0} - beta * omega, &v);  // p = r + beta (p - omega v)
      prec(p, ph);
      Dop(ph, v);
      const cx<double> rv = fdots(g, {{&rh, &v}})[0];
      const double rv2 = rv.r * rv.r + rv.i * rv.i;
      if (!(rv2 > 0.0)) {
        breakdown = true;
        break;
      }
      alpha = rho_new * cx<double>{1.0 / rv2, 0} * conj(rv);
      faxpy(g, one, r, zero, sv, cx<double>{0, 0} - alpha, &v);  // s = r - alpha v
      prec(sv, sh);
      Dop(sh, t);
      auto d = fdots(g, {{&t, &sv}, {&t, &t}});
      omega = d[1].r > 0 ? d[0] * cx<double>{1.0 / d[1].r, 0} : zero;
      faxpy(g, alpha, ph, one, x, omega, &sh);                    // x += alpha p^ + omega s^
      faxpy(g, one, sv, zero, r, cx<double>{0, 0} - omega, &t);   // r = s - omega t
      r2 = fdots(g, {{&r, &r}})[0].r;
      rho = rho_new;
      info.inner_iters += 1;
      if (omega.r == 0.0 && omega.i == 0.0) {
        breakdown = true;
        break;
      }
    }
    if (breakdown) info.restarts += 1;
  }
  if (status != BRIDGE_OK) {
    Dop(x, t);
    faxpy(g, one, b, zero, r, cx<double>{-1, 0}, &t);
    const double r2 = fdots(g, {{&r, &r}})[0].r;
    info.true_rel_residual = std::sqrt(r2 / b2);
    if (r2 <= tol2) status = BRIDGE_OK;
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
  p->sap_cycles = 2;
  p->mr_steps = 4;
  p->coarse_tol = 5e-2;
  p->coarse_maxiter = 200;
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

int bridge_mg_info(bridge_mg g, int* nblocks, int* nvec) {
  if (!g) return BRIDGE_EINVAL;
  if (nblocks) *nblocks = g->m.nblocks;
  if (nvec) *nvec = g->nv;
  return BRIDGE_OK;
}

}  // extern "C"
