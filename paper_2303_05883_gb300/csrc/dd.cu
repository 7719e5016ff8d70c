// Domain decomposition of the lattice along t with a halo exchange between
// the sub-domains, the paper's way of spreading one lattice over nodes
// (Sec. 2: the lattice is divided among MPI processes, each of which
// exchanges the boundary data of its sub-lattice with its neighbours through
// persistent communication while the bulk is computed; Sec. 3: weak and
// strong scaling over such decompositions).
//
// The global lattice is cut into nparts slabs of Lt / nparts time slices.
// Each slab is a sub-lattice of its own (links, clover term and fields in
// the GPU layout of its local extents, its own stream).  Every slab starts at
// an even time slice, so the even-odd parity of a site is the same locally
// and globally, and because t is the slowest index, a slab's part of a
// canonical field is one contiguous range per right-hand side.
//
// One application of a hopping term (D_eo, D_oe, either pass of the Schur
// operator of Eq. 1, the full operator) runs in three overlapping parts:
//   * interior: the ordinary stencil on the slab with the boundary phase of
//     the t direction set to zero, i.e. every t hop that would leave the slab
//     contributes nothing (all fused epilogues included);
//   * faces, on a second stream per slab: the spin-projected two-component
//     half spinors of the first time slice ((1 - gamma_t) psi, for the
//     forward hops of the slab below) and, of the last time slice, the
//     projected half spinors already multiplied by U_t^dagger (for the
//     backward hops of the slab above) -- 6 complex numbers per face site
//     instead of 12 -- are packed and copied into the neighbours' receive
//     buffers;
//   * boundary: once both neighbours' faces have arrived, the contributions
//     of the t hops across the slab boundary are reconstructed to four spin
//     components (the forward ones multiplied by the receiver's own link),
//     multiplied by beta, by the global boundary phase where the hop wraps
//     the lattice and, with a T^-1 epilogue, by T^-1 at the site (the
//     epilogues are linear), and added to the interior result.
// Global scalars (the dot products of the solver) are sums of per-slab
// partial sums: the all-reduce of the decomposed solver.
//
// The transport between slabs is a device-to-device copy: here the slabs
// share one GPU.  The clover term is built once from the whole gauge field
// and each slab receives its part.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include "host.h"

using namespace bridge;

// ------------------------------------------------------------- face kernels
namespace bridge {

struct DdFaceArgs {
  long vh;           // sites per parity of the slab
  uint32_t nface;    // sites per parity of one time slice (Lx Ly Lz / 2)
  int lt;            // time slices of the slab
  int nrhs;
  int q;             // parity of the input sites (the output parity is 1 - q)
  const char* in;    // input field block of parity q, rhs 0
  long in_rs;
  const char* gauge;  // the slab's links [parity][mu]
  void* up;          // packed (1 - gamma_t) psi of slice 0: [rhs][6][nface]
  void* dn;          // packed U_t^dag (1 + gamma_t) psi of slice lt - 1
};

// Thread (face site f, right-hand side): both faces of that site.
template <int P>
__global__ void __launch_bounds__(256) k_dd_pack(const DdFaceArgs a) {
  using R = typename Tr<P>::R;
  const long n = (long)a.nface * a.nrhs;
  for (long t = (long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long)gridDim.x * blockDim.x) {
    const int rhs = (int)(t / a.nface);
    const uint32_t f = (uint32_t)(t % a.nface);
    const char* in = a.in + rhs * a.in_rs;
    cx<R>* up = reinterpret_cast<cx<R>*>(a.up) + (long)rhs * 6 * a.nface;
    cx<R>* dn = reinterpret_cast<cx<R>*>(a.dn) + (long)rhs * 6 * a.nface;
    {
      // first slice: the forward t hop of the slab below reads (1 - gamma_t) psi here
      cx<R> psi[12], h[2][3];
      load_spinor<P>(in, a.vh, f, psi);
      project<R, 3, true>(psi, h);
#pragma unroll
      for (int k = 0; k < 2; ++k)
#pragma unroll
        for (int c = 0; c < 3; ++c) up[(k * 3 + c) * (long)a.nface + f] = h[k][c];
    }
    {
      // last slice: the backward t hop of the slab above reads U_t^dag (1 + gamma_t) psi
      const uint32_t ih = (uint32_t)(a.lt - 1) * a.nface + f;
      cx<R> psi[12], h[2][3];
      load_spinor<P>(in, a.vh, ih, psi);
      project<R, 3, false>(psi, h);
      const long lbb = link_block_bytes(P, a.vh);
      Link<R> U;
      load_link<P>(a.gauge + ((long)a.q * 4 + 3) * lbb, a.vh, ih, U);
#pragma unroll
      for (int k = 0; k < 2; ++k)
#pragma unroll
        for (int r = 0; r < 3; ++r)
          dn[(k * 3 + r) * (long)a.nface + f] = crow3_conj(U.m[0][r], U.m[1][r], U.m[2][r], h[k]);
    }
  }
}

struct DdBoundaryArgs {
  long vh;
  uint32_t nface;
  int lt, nrhs;
  int p;                 // output parity
  char* out;             // output field block of parity p, rhs 0 (read, added to, written)
  long out_rs;
  const char* gauge;     // the slab's links
  const char* clovE;     // T^-1 blocks [parity] (null: no T^-1 epilogue)
  const void* from_up;   // the slab above's first-slice face: [rhs][6][nface]
  const void* from_dn;   // the slab below's last-slice face
  double beta_up, beta_dn;  // beta times the boundary phase of each crossing
};

// Thread (face site f, side, right-hand side): side 0 = the slab's last
// slice (forward t hop into the slab above), side 1 = its first slice
// (backward t hop into the slab below).
template <int P, bool ECLOV>
__global__ void __launch_bounds__(256) k_dd_boundary(const DdBoundaryArgs a) {
  using R = typename Tr<P>::R;
  const long n = 2L * a.nface * a.nrhs;
  for (long t = (long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long)gridDim.x * blockDim.x) {
    const int rhs = (int)(t / (2L * a.nface));
    const int side = (int)((t / a.nface) & 1);
    const uint32_t f = (uint32_t)(t % a.nface);
    const uint32_t ih = side == 0 ? (uint32_t)(a.lt - 1) * a.nface + f : f;
    cx<R> acc[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) acc[k] = czero<R>();
    if (side == 0) {
      const cx<R>* h = reinterpret_cast<const cx<R>*>(a.from_up) + (long)rhs * 6 * a.nface;
      cx<R> hh[2][3], u[2][3];
#pragma unroll
      for (int k = 0; k < 2; ++k)
#pragma unroll
        for (int c = 0; c < 3; ++c) hh[k][c] = h[(k * 3 + c) * (long)a.nface + f];
      const long lbb = link_block_bytes(P, a.vh);
      Link<R> U;
      load_link<P>(a.gauge + ((long)a.p * 4 + 3) * lbb, a.vh, ih, U);
#pragma unroll
      for (int k = 0; k < 2; ++k)
#pragma unroll
        for (int r = 0; r < 3; ++r) u[k][r] = crow3(U.m[r][0], U.m[r][1], U.m[r][2], hh[k]);
      reconstruct<R, 3, true>(u, acc);
#pragma unroll
      for (int k = 0; k < 12; ++k) acc[k] = (R)a.beta_up * acc[k];
    } else {
      const cx<R>* h = reinterpret_cast<const cx<R>*>(a.from_dn) + (long)rhs * 6 * a.nface;
      cx<R> u[2][3];
#pragma unroll
      for (int k = 0; k < 2; ++k)
#pragma unroll
        for (int c = 0; c < 3; ++c) u[k][c] = h[(k * 3 + c) * (long)a.nface + f];
      reconstruct<R, 3, false>(u, acc);
#pragma unroll
      for (int k = 0; k < 12; ++k) acc[k] = (R)a.beta_dn * acc[k];
    }
    cx<R> v[12];
    if constexpr (ECLOV) {
      clover_apply<P>(a.clovE + (long)a.p * clover_block_bytes(P, a.vh), a.vh, ih, acc, v);
    } else {
#pragma unroll
      for (int k = 0; k < 12; ++k) v[k] = acc[k];
    }
    char* out = a.out + rhs * a.out_rs;
    cx<R> o[12];
    load_spinor<P, false>(out, a.vh, ih, o);
#pragma unroll
    for (int k = 0; k < 12; ++k) o[k] = o[k] + v[k];
    store_spinor<P>(out, a.vh, ih, o);
  }
}

// ------------------------------------------------------ FP64 vector kernels
// out = c0 v0 + c1 v1 + c2 v2 over the 24 reals of every site (inputs may
// alias out; a null input is skipped), and block partials of
// (Re <a, b>, Im <a, b>, |b|^2) for the decomposed BiCGStab.
struct DdVecArgs {
  long n;  // double2 entries (12 per site)
  double2* out;
  const double2* v[3];
  double c[3][2];
};
__global__ void __launch_bounds__(256) k_dd_lincomb(const DdVecArgs a) {
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += (long)gridDim.x * blockDim.x) {
    cx<double> s = czero<double>();
#pragma unroll
    for (int k = 0; k < 3; ++k)
      if (a.v[k]) {
        const double2 x = a.v[k][i];
        s = cfma(cx<double>{a.c[k][0], a.c[k][1]}, cx<double>{x.x, x.y}, s);
      }
    a.out[i] = make_double2(s.r, s.i);
  }
}
__global__ void __launch_bounds__(256) k_dd_dot(const double2* x, const double2* y, long n, double* partials) {
  __shared__ double sh[32][4];
  double v[3] = {0.0, 0.0, 0.0};
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const double2 a = x[i], b = y[i];
    v[0] += a.x * b.x + a.y * b.y;
    v[1] += a.x * b.y - a.y * b.x;
    v[2] += b.x * b.x + b.y * b.y;
  }
  block_sum<3>(v, sh);
  if (threadIdx.x == 0)
    for (int k = 0; k < 3; ++k) partials[blockIdx.x * 3 + k] = v[k];
}

}  // namespace bridge

// ------------------------------------------------------------- host side
struct bridge_dd_s {
  bridge_lattice_s* global = nullptr;
  bridge_op op{};
  int nparts = 1, lt = 0;
  long vs = 0;          // sites of one time slice
  uint32_t nface = 0;   // vs / 2
  struct Slab {
    bridge_lattice_s* L = nullptr;
    int t0 = 0;
    cudaStream_t comm = nullptr;
    cudaEvent_t ev_in = nullptr, ev_sent = nullptr, ev_done = nullptr;
    std::unique_ptr<DevBuf> send_up, send_dn, recv_up, recv_dn;  // faces
    size_t face_bytes = 0;
  };
  std::vector<Slab> slabs;
  std::unique_ptr<DevBuf> dots;  // per-slab block partials of the dot products
  std::vector<double> hdots;
};

namespace {

constexpr int kDotBlocks = 64;

void slab_plan(const int dims[4], int nparts, int rank, bridge_dd_plan* pl) {
  std::memset(pl, 0, sizeof(*pl));
  const int lt = dims[3] / nparts;
  for (int k = 0; k < 3; ++k) pl->local_dims[k] = dims[k];
  pl->local_dims[3] = lt;
  pl->t0 = rank * lt;
  pl->rank_up = (rank + 1) % nparts;
  pl->rank_down = (rank + nparts - 1) % nparts;
  pl->face_sites = (long)dims[0] * dims[1] * dims[2] / 2;
  pl->up_wraps = rank == nparts - 1;
  pl->down_wraps = rank == 0;
  pl->canon_offset_sites = (long)pl->t0 * dims[0] * dims[1] * dims[2];
}

void check_plan_args(const int dims[4], int nparts) {
  BR_CHECK(dims != nullptr, BRIDGE_EINVAL, "NULL dims");
  for (int k = 0; k < 4; ++k) BR_CHECK(dims[k] >= 2 && dims[k] % 2 == 0, BRIDGE_EINVAL, "extents must be even and >= 2");
  BR_CHECK(nparts >= 1 && dims[3] % nparts == 0 && (dims[3] / nparts) % 2 == 0, BRIDGE_EINVAL,
           "nparts must divide Lt into slabs of an even number (>= 2) of time slices");
}

// Copy a [planes][vh] block of the global lattice (16-byte planes) to the
// slab's [planes][vh_loc] block: one contiguous run per plane.
void copy_planes(char* dst, long vh_loc, const char* src, long vh, long first, int planes, cudaStream_t st) {
  BR_CUDA(cudaMemcpy2DAsync(dst, (size_t)vh_loc * 16, src + first * 16, (size_t)vh * 16, (size_t)vh_loc * 16,
                            (size_t)planes, cudaMemcpyDeviceToDevice, st));
}

void ensure_faces(bridge_dd_s* d, int prec, int nrhs) {
  const size_t need = (size_t)nrhs * 6 * d->nface * (prec == P_F64 ? 16 : 8);
  for (auto& s : d->slabs)
    if (s.face_bytes < need) {
      s.send_up.reset(new DevBuf(need));
      s.send_dn.reset(new DevBuf(need));
      s.recv_up.reset(new DevBuf(need));
      s.recv_dn.reset(new DevBuf(need));
      s.face_bytes = need;
    }
}

template <int P>
void launch_pack(const DdFaceArgs& a, cudaStream_t st) {
  const long n = (long)a.nface * a.nrhs;
  const unsigned grid = (unsigned)std::min<long>((n + 255) / 256, 8L * sm_count());
  k_dd_pack<P><<<grid, 256, 0, st>>>(a);
}
template <int P>
void launch_boundary(const DdBoundaryArgs& a, cudaStream_t st) {
  const long n = 2L * a.nface * a.nrhs;
  const unsigned grid = (unsigned)std::min<long>((n + 255) / 256, 8L * sm_count());
  if (a.clovE)
    k_dd_boundary<P, true><<<grid, 256, 0, st>>>(a);
  else
    k_dd_boundary<P, false><<<grid, 256, 0, st>>>(a);
}
#define DD_PREC_CALL(prec, FN, ...)                   \
  switch (prec) {                                     \
    case P_F64: FN<P_F64>(__VA_ARGS__); break;        \
    case P_F32: FN<P_F32>(__VA_ARGS__); break;        \
    case P_F16: FN<P_F16>(__VA_ARGS__); break;        \
    default: FN<P_BF16>(__VA_ARGS__); break;          \
  }

// One hop term on every slab: out_s = epilogue(beta H in_s + ...) with the
// t hops across slab boundaries taken from the neighbours' faces.  `base`
// carries flags, coefficients and the reduction-free call; per-slab fields
// come from the lambdas.  Queued on the slabs' streams; the caller joins.
template <class FieldsFn>
void dd_hop(bridge_dd_s* d, HopCall base, int prec, int nrhs, FieldsFn fields) {
  const int p = base.out_parity, q = 1 - p;
  const int R = d->nparts;
  if (R > 1) ensure_faces(d, prec, nrhs);
  // every slab's inputs (and its previous boundary update) are complete
  for (auto& s : d->slabs) BR_CUDA(cudaEventRecord(s.ev_in, s.L->stream));
  for (int r = 0; r < R; ++r) {
    auto& s = d->slabs[r];
    HopCall c = base;
    fields(r, c);
    if (R > 1) c.bc[3] = 0;  // t hops leaving the slab: from the faces
    if (R > 1) {
      // faces on the second stream, overlapping the interior stencil
      auto& up = d->slabs[(r + 1) % R];
      auto& dn = d->slabs[(r + R - 1) % R];
      BR_CUDA(cudaStreamWaitEvent(s.comm, s.ev_in, 0));
      BR_CUDA(cudaStreamWaitEvent(s.comm, up.ev_in, 0));  // its receive buffer is free
      BR_CUDA(cudaStreamWaitEvent(s.comm, dn.ev_in, 0));
      DdFaceArgs fa;
      std::memset(&fa, 0, sizeof(fa));
      fa.vh = s.L->vh;
      fa.nface = d->nface;
      fa.lt = d->lt;
      fa.nrhs = nrhs;
      fa.q = q;
      fa.in = c.in;
      fa.in_rs = c.in_rs;
      fa.gauge = gauge_ptr(s.L, prec);
      fa.up = s.send_up->ptr;
      fa.dn = s.send_dn->ptr;
      note_launch(s.L, K_HOP, 0, 0, s.comm, true);
      DD_PREC_CALL(prec, launch_pack, fa, s.comm);
      note_launch(s.L, K_HOP, 0, 0, s.comm, false);
      BR_CUDA(cudaGetLastError());
      const size_t bytes = (size_t)nrhs * 6 * d->nface * (prec == P_F64 ? 16 : 8);
      // the first slice goes to the slab below (its forward hops), the last to the slab above
      BR_CUDA(cudaMemcpyAsync(dn.recv_up->ptr, s.send_up->ptr, bytes, cudaMemcpyDeviceToDevice, s.comm));
      BR_CUDA(cudaMemcpyAsync(up.recv_dn->ptr, s.send_dn->ptr, bytes, cudaMemcpyDeviceToDevice, s.comm));
      BR_CUDA(cudaEventRecord(s.ev_sent, s.comm));
    }
    run_hop(s.L, c, s.L->stream);
  }
  if (R == 1) return;
  for (int r = 0; r < R; ++r) {
    auto& s = d->slabs[r];
    auto& up = d->slabs[(r + 1) % R];
    auto& dn = d->slabs[(r + R - 1) % R];
    BR_CUDA(cudaStreamWaitEvent(s.L->stream, up.ev_sent, 0));
    BR_CUDA(cudaStreamWaitEvent(s.L->stream, dn.ev_sent, 0));
    HopCall c = base;
    fields(r, c);
    DdBoundaryArgs ba;
    std::memset(&ba, 0, sizeof(ba));
    ba.vh = s.L->vh;
    ba.nface = d->nface;
    ba.lt = d->lt;
    ba.nrhs = nrhs;
    ba.p = p;
    ba.out = c.out;
    ba.out_rs = c.out_rs;
    ba.gauge = gauge_ptr(s.L, prec);
    ba.clovE = (c.flags & F_E_CLOV) ? clover_ptr(s.L, prec, true, c.kcsw) : nullptr;
    ba.from_up = s.recv_up->ptr;
    ba.from_dn = s.recv_dn->ptr;
    ba.beta_up = c.beta * (r == R - 1 ? d->op.bc[3] : 1);
    ba.beta_dn = c.beta * (r == 0 ? d->op.bc[3] : 1);
    note_launch(s.L, K_HOP, 0, 0, s.L->stream, true);
    DD_PREC_CALL(prec, launch_boundary, ba, s.L->stream);
    note_launch(s.L, K_HOP, 0, 0, s.L->stream, false);
    BR_CUDA(cudaGetLastError());
  }
}

// Wait on the global stream for every slab's queued work.
void dd_join(bridge_dd_s* d) {
  for (auto& s : d->slabs) {
    BR_CUDA(cudaEventRecord(s.ev_done, s.L->stream));
    BR_CUDA(cudaStreamWaitEvent(d->global->stream, s.ev_done, 0));
  }
}
// The slabs wait for the global stream (inputs written there).
void dd_fork(bridge_dd_s* d) {
  cudaEvent_t e = d->slabs[0].ev_done;
  BR_CUDA(cudaEventRecord(e, d->global->stream));
  for (auto& s : d->slabs) BR_CUDA(cudaStreamWaitEvent(s.L->stream, e, 0));
}

// Per-slab fields of one kind (workspace of each sub-lattice).
std::vector<Field> dd_fields(bridge_dd_s* d, const std::string& name, int prec, int subset, int nrhs) {
  std::vector<Field> v;
  for (auto& s : d->slabs) v.push_back(workspace(s.L, "dd_" + name, prec, subset, nrhs));
  return v;
}

// Canonical FP64 device arrays <-> per-slab fields: whole-lattice fields
// (subset FULL) or half-lattice vectors of one parity.  A slab's part of a
// canonical array starts at its first time slice; right-hand sides keep the
// global stride.
void dd_import(bridge_dd_s* d, const double* canon, const std::vector<Field>& f) {
  const bool full = f[0].subset == BRIDGE_FULL;
  const long vg = full ? d->global->V : d->global->vh;
  for (int r = 0; r < d->nparts; ++r) {
    auto& s = d->slabs[r];
    const long off = (long)s.t0 * (full ? d->vs : (long)d->nface);
    canon_to_field(s.L, canon + off * 24, f[r], s.L->stream, nullptr, vg * 24);
  }
}
void dd_export(bridge_dd_s* d, const std::vector<Field>& f, double* canon) {
  const bool full = f[0].subset == BRIDGE_FULL;
  const long vg = full ? d->global->V : d->global->vh;
  for (int r = 0; r < d->nparts; ++r) {
    auto& s = d->slabs[r];
    const long off = (long)s.t0 * (full ? d->vs : (long)d->nface);
    field_to_canon(s.L, f[r], canon + off * 24, s.L->stream, vg * 24);
  }
}

HopCall dd_call(bridge_dd_s* d, int prec, int nrhs) {
  HopCall c;
  c.prec = prec;
  c.nrhs = nrhs;
  c.kcsw = op_kcsw(d->op);
  for (int k = 0; k < 4; ++k) c.bc[k] = d->op.bc[k];
  return c;
}

// D_eo (q = 0) / D_oe (q = 1): out (parity q) = -kappa H in (parity 1 - q)
void dd_deo(bridge_dd_s* d, int prec, int q, const std::vector<Field>& out, const std::vector<Field>& in) {
  HopCall c = dd_call(d, prec, out[0].nrhs);
  c.out_parity = q;
  c.beta = -d->op.kappa;
  dd_hop(d, c, prec, out[0].nrhs, [&](int r, HopCall& h) {
    h.out = out[r].ptr(q);
    h.out_rs = out[r].rs;
    h.in = in[r].ptr(1 - q);
    h.in_rs = in[r].rs;
  });
}

// Full operator: out = T in - kappa H in, one hop term per output parity.
void dd_d(bridge_dd_s* d, int prec, const std::vector<Field>& out, const std::vector<Field>& in) {
  for (int q = 0; q < 2; ++q) {
    HopCall c = dd_call(d, prec, out[0].nrhs);
    c.flags = F_SELF | (op_is_clover(d->op) ? F_SELF_CLOV : 0);
    c.cls = K_FULLD;
    c.out_parity = q;
    c.beta = -d->op.kappa;
    c.s1 = 1.0;
    dd_hop(d, c, prec, out[0].nrhs, [&](int r, HopCall& h) {
      h.out = out[r].ptr(q);
      h.out_rs = out[r].rs;
      h.in = in[r].ptr(1 - q);
      h.in_rs = in[r].rs;
      h.self = in[r].ptr(q);
      h.self_rs = in[r].rs;
    });
  }
}

// Schur operator of Eq. 1 on even fields: tmp_o = T_oo^-1 (-kappa H_oe in_e),
// out_e = in_e - T_ee^-1 (-kappa H_eo tmp_o).
void dd_dhat(bridge_dd_s* d, int prec, const std::vector<Field>& out, const std::vector<Field>& in,
             const std::vector<Field>& tmp) {
  const bool clov = op_is_clover(d->op);
  HopCall c = dd_call(d, prec, out[0].nrhs);
  c.flags = clov ? F_E_CLOV : 0;
  c.cls = K_DHAT1;
  c.out_parity = 1;
  c.beta = -d->op.kappa;
  dd_hop(d, c, prec, out[0].nrhs, [&](int r, HopCall& h) {
    h.out = tmp[r].ptr(1);
    h.out_rs = tmp[r].rs;
    h.in = in[r].ptr(0);
    h.in_rs = in[r].rs;
  });
  c.flags = F_SELF | (clov ? F_E_CLOV : 0);
  c.cls = K_DHAT2;
  c.out_parity = 0;
  c.beta = d->op.kappa;
  c.s1 = 1.0;
  dd_hop(d, c, prec, out[0].nrhs, [&](int r, HopCall& h) {
    h.out = out[r].ptr(0);
    h.out_rs = out[r].rs;
    h.in = tmp[r].ptr(1);
    h.in_rs = tmp[r].rs;
    h.self = in[r].ptr(0);
    h.self_rs = in[r].rs;
  });
}

// Even-odd source preparation and reconstruction (FP64, one right-hand side):
// out_q = T_qq^-1 (src_q + kappa H_q,1-q v_{1-q}), v = T_oo^-1 b_o for the
// preparation (q = 0) or the even solution (q = 1).
void dd_prep(bridge_dd_s* d, int q, const std::vector<Field>& out, const std::vector<Field>& v,
             const std::vector<Field>& src) {
  const bool clov = op_is_clover(d->op);
  HopCall c = dd_call(d, P_F64, 1);
  c.flags = F_AUX | (clov ? F_E_CLOV : 0);
  c.cls = K_PREP;
  c.out_parity = q;
  c.beta = d->op.kappa;
  c.caux = 1.0;
  dd_hop(d, c, P_F64, 1, [&](int r, HopCall& h) {
    h.out = out[r].ptr(q);
    h.out_rs = out[r].rs;
    h.in = v[r].ptr(1 - q);
    h.in_rs = v[r].rs;
    h.aux = src[r].ptr(q);
    h.aux_rs = src[r].rs;
  });
}

// ---- the decomposed BiCGStab's vector algebra (FP64 even fields, 1 rhs)
struct Vec {
  const std::vector<Field>* f;
  int parity;
};
double2* vp(const Vec& v, int r) { return reinterpret_cast<double2*>((*v.f)[r].ptr(v.parity)); }

void lincomb(bridge_dd_s* d, const Vec& out, std::initializer_list<std::pair<cx<double>, Vec>> terms) {
  for (int r = 0; r < d->nparts; ++r) {
    auto& s = d->slabs[r];
    DdVecArgs a;
    std::memset(&a, 0, sizeof(a));
    a.n = s.L->vh * 12;
    a.out = vp(out, r);
    int k = 0;
    for (const auto& t : terms) {
      a.v[k] = vp(t.second, r);
      a.c[k][0] = t.first.r;
      a.c[k][1] = t.first.i;
      ++k;
    }
    const unsigned grid = (unsigned)std::min<long>((a.n + 255) / 256, 4L * sm_count());
    note_launch(s.L, K_BLAS_XR, (double)s.L->vh * 192 * (k + 1), 0, s.L->stream, true);
    k_dd_lincomb<<<grid, 256, 0, s.L->stream>>>(a);
    note_launch(s.L, K_BLAS_XR, 0, 0, s.L->stream, false);
    BR_CUDA(cudaGetLastError());
  }
}

// (<a, b>, |b|^2) over the whole lattice: per-slab block partials, then the
// sum over blocks and slabs on the host (the all-reduce).
void dots(bridge_dd_s* d, const Vec& a, const Vec& b, cx<double>& ab, double& bb) {
  const size_t need = (size_t)d->nparts * kDotBlocks * 3;
  if (!d->dots || d->dots->bytes < need * sizeof(double)) d->dots.reset(new DevBuf(need * sizeof(double)));
  for (int r = 0; r < d->nparts; ++r) {
    auto& s = d->slabs[r];
    note_launch(s.L, K_NORM, (double)s.L->vh * 384, 0, s.L->stream, true);
    k_dd_dot<<<kDotBlocks, 256, 0, s.L->stream>>>(vp(a, r), vp(b, r), s.L->vh * 12,
                                                 reinterpret_cast<double*>(d->dots->ptr) + (size_t)r * kDotBlocks * 3);
    note_launch(s.L, K_NORM, 0, 0, s.L->stream, false);
    BR_CUDA(cudaGetLastError());
  }
  dd_join(d);
  d->hdots.resize(need);
  BR_CUDA(cudaMemcpyAsync(d->hdots.data(), d->dots->ptr, need * sizeof(double), cudaMemcpyDeviceToHost,
                          d->global->stream));
  BR_CUDA(cudaStreamSynchronize(d->global->stream));
  double s0 = 0, s1 = 0, s2 = 0;
  for (size_t i = 0; i < need; i += 3) {
    s0 += d->hdots[i];
    s1 += d->hdots[i + 1];
    s2 += d->hdots[i + 2];
  }
  ab = {s0, s1};
  bb = s2;
}

cx<double> zdivd(cx<double> a, cx<double> b) {
  const double n = b.r * b.r + b.i * b.i;
  return {(a.r * b.r + a.i * b.i) / n, (a.i * b.r - a.r * b.i) / n};
}

}  // namespace

// ------------------------------------------------------------------- C-ABI
#define DD_BEGIN try {
#define DD_END                   \
  }                              \
  catch (const Error& e) {       \
    set_error(e.code, e.msg);    \
    return e.code;               \
  }                              \
  catch (const std::bad_alloc&) { \
    set_error(BRIDGE_ENOMEM, "host allocation"); \
    return BRIDGE_ENOMEM;        \
  }                              \
  return BRIDGE_OK;

extern "C" int bridge_dd_plan_of(const int dims[4], int nparts, int rank, bridge_dd_plan* plan) {
  DD_BEGIN
  BR_CHECK(plan != nullptr, BRIDGE_EINVAL, "NULL plan");
  check_plan_args(dims, nparts);
  BR_CHECK(rank >= 0 && rank < nparts, BRIDGE_EINVAL, "rank out of range");
  slab_plan(dims, nparts, rank, plan);
  DD_END
}

extern "C" int bridge_dd_create(bridge_lattice L, const bridge_op* op, int nparts, bridge_dd* out) {
  DD_BEGIN
  BR_CHECK(L != nullptr && op != nullptr && out != nullptr, BRIDGE_EINVAL, "NULL argument");
  *out = nullptr;
  BR_CHECK(op->kind == BRIDGE_WILSON || op->kind == BRIDGE_CLOVER, BRIDGE_EINVAL, "op.kind: WILSON or CLOVER");
  for (int k = 0; k < 4; ++k) BR_CHECK(op->bc[k] == 1 || op->bc[k] == -1, BRIDGE_EINVAL, "op.bc must be +1 or -1");
  check_plan_args(L->dims, nparts);
  BR_CHECK(L->have_gauge, BRIDGE_ESTATE, "no gauge field uploaded");
  std::lock_guard<std::mutex> lk(L->api_mu);
  std::unique_ptr<bridge_dd_s> d(new bridge_dd_s());
  d->global = L;
  d->op = *op;
  d->nparts = nparts;
  d->lt = L->dims[3] / nparts;
  d->vs = (long)L->dims[0] * L->dims[1] * L->dims[2];
  d->nface = (uint32_t)(d->vs / 2);
  const bool clov = op_is_clover(*op);
  std::shared_ptr<CloverSet> gset;
  if (clov) gset = clover_set(L, op_kcsw(*op));  // the term of the whole field
  BR_CUDA(cudaStreamSynchronize(L->stream));
  d->slabs.resize(nparts);
  for (int r = 0; r < nparts; ++r) {
    auto& s = d->slabs[r];
    bridge_dd_plan pl;
    slab_plan(L->dims, nparts, r, &pl);
    s.t0 = pl.t0;
    const int st = bridge_lattice_create(pl.local_dims, &s.L);
    if (st != BRIDGE_OK) throw Error{st, "slab lattice"};
    BR_CUDA(cudaStreamCreateWithFlags(&s.comm, cudaStreamNonBlocking));
    BR_CUDA(cudaEventCreateWithFlags(&s.ev_in, cudaEventDisableTiming));
    BR_CUDA(cudaEventCreateWithFlags(&s.ev_sent, cudaEventDisableTiming));
    BR_CUDA(cudaEventCreateWithFlags(&s.ev_done, cudaEventDisableTiming));
    const long vh = L->vh, vhl = s.L->vh, first = (long)s.t0 * d->nface;
    // links: [parity][mu] blocks of 9 double2 planes
    s.L->gauge[P_F64].reset(new DevBuf((size_t)(8 * link_block_bytes(P_F64, vhl))));
    for (int b = 0; b < 8; ++b)
      copy_planes(s.L->gauge[P_F64]->ptr + b * link_block_bytes(P_F64, vhl), vhl,
                  L->gauge[P_F64]->ptr + b * link_block_bytes(P_F64, vh), vh, first, 9, s.L->stream);
    s.L->have_gauge = true;
    if (clov) {
      // the slab's part of T and T^-1 of the whole field: [parity] blocks of 36 double2 planes
      auto cs = std::make_shared<CloverSet>();
      cs->kcsw = op_kcsw(*op);
      for (int inv = 0; inv < 2; ++inv) {
        std::unique_ptr<DevBuf>& dst = inv ? cs->Tinv[P_F64] : cs->T[P_F64];
        const DevBuf& src = inv ? *gset->Tinv[P_F64] : *gset->T[P_F64];
        dst.reset(new DevBuf((size_t)(2 * clover_block_bytes(P_F64, vhl))));
        for (int p = 0; p < 2; ++p)
          copy_planes(dst->ptr + p * clover_block_bytes(P_F64, vhl), vhl, src.ptr + p * clover_block_bytes(P_F64, vh),
                      vh, first, 36, s.L->stream);
      }
      std::lock_guard<std::mutex> lc(s.L->clover_mu);
      s.L->clovers.insert(s.L->clovers.begin(), cs);
    }
    BR_CUDA(cudaStreamSynchronize(s.L->stream));
  }
  *out = d.release();
  DD_END
}

extern "C" int bridge_dd_destroy(bridge_dd d) {
  DD_BEGIN
  if (!d) return BRIDGE_OK;
  for (auto& s : d->slabs) {
    if (s.L) cudaStreamSynchronize(s.L->stream);
    if (s.comm) {
      cudaStreamSynchronize(s.comm);
      cudaStreamDestroy(s.comm);
    }
    for (cudaEvent_t e : {s.ev_in, s.ev_sent, s.ev_done})
      if (e) cudaEventDestroy(e);
    s.send_up.reset();
    s.send_dn.reset();
    s.recv_up.reset();
    s.recv_dn.reset();
    if (s.L) bridge_lattice_destroy(s.L);
  }
  delete d;
  DD_END
}

// which: 0 full D, 1 D_eo / D_oe (out_parity), 2 the Schur operator.
static int dd_mult(bridge_dd d, int prec, int which, int out_parity, const double* in, double* out, int nrhs) {
  DD_BEGIN
  BR_CHECK(d != nullptr, BRIDGE_EINVAL, "NULL handle");
  BR_CHECK(prec >= BRIDGE_F64 && prec <= BRIDGE_BF16, BRIDGE_EINVAL, "precision");
  BR_CHECK(nrhs >= 0, BRIDGE_EINVAL, "nrhs < 0");
  if (nrhs == 0) return BRIDGE_OK;
  BR_CHECK(in != nullptr && out != nullptr, BRIDGE_EINVAL, "in/out is NULL");
  BR_CHECK(out_parity == 0 || out_parity == 1, BRIDGE_EINVAL, "out_parity");
  std::lock_guard<std::mutex> lk(d->global->api_mu);
  dd_fork(d);
  if (which == 0) {
    auto fin = dd_fields(d, "in", prec, BRIDGE_FULL, nrhs), fout = dd_fields(d, "out", prec, BRIDGE_FULL, nrhs);
    dd_import(d, in, fin);
    dd_d(d, prec, fout, fin);
    dd_export(d, fout, out);
  } else if (which == 1) {
    const int q = out_parity;
    auto fin = dd_fields(d, "hin", prec, 1 - q, nrhs), fout = dd_fields(d, "hout", prec, q, nrhs);
    dd_import(d, in, fin);
    dd_deo(d, prec, q, fout, fin);
    dd_export(d, fout, out);
  } else {
    auto fin = dd_fields(d, "hin", prec, BRIDGE_EVEN, nrhs), fout = dd_fields(d, "hout", prec, BRIDGE_EVEN, nrhs),
         ftmp = dd_fields(d, "htmp", prec, BRIDGE_ODD, nrhs);
    dd_import(d, in, fin);
    dd_dhat(d, prec, fout, fin, ftmp);
    dd_export(d, fout, out);
  }
  dd_join(d);
  BR_CUDA(cudaStreamSynchronize(d->global->stream));
  DD_END
}

extern "C" int bridge_dd_mult_D_dev(bridge_dd d, int prec, const double* in, double* out, int nrhs) {
  return dd_mult(d, prec, 0, 0, in, out, nrhs);
}
extern "C" int bridge_dd_mult_Deo_dev(bridge_dd d, int prec, int out_parity, const double* in, double* out, int nrhs) {
  return dd_mult(d, prec, 1, out_parity, in, out, nrhs);
}
extern "C" int bridge_dd_mult_Dhat_dev(bridge_dd d, int prec, const double* in, double* out, int nrhs) {
  return dd_mult(d, prec, 2, 0, in, out, nrhs);
}

// Plain FP64 BiCGStab on the even-odd system over the slabs (every dot
// product reduced over all slabs), with the even-odd preparation and
// reconstruction and the FP64 true residual of the whole lattice.
extern "C" int bridge_dd_solve_dev(bridge_dd d, const bridge_solver* prm, const double* b_dev, double* x_dev,
                                   int nrhs, bridge_info* info) {
  DD_BEGIN
  BR_CHECK(d != nullptr && prm != nullptr, BRIDGE_EINVAL, "NULL argument");
  BR_CHECK(nrhs >= 0, BRIDGE_EINVAL, "nrhs < 0");
  if (nrhs == 0) return BRIDGE_OK;
  BR_CHECK(b_dev != nullptr && x_dev != nullptr && info != nullptr, BRIDGE_EINVAL, "NULL buffer");
  BR_CHECK(prm->tol > 0, BRIDGE_EINVAL, "tol");
  std::lock_guard<std::mutex> lk(d->global->api_mu);
  const auto t0 = std::chrono::steady_clock::now();
  const bool clov = op_is_clover(d->op);
  const long V = d->global->V;
  const int max_iter = prm->max_iter > 0 ? prm->max_iter : 20000;
  auto B = dd_fields(d, "sB", P_F64, BRIDGE_FULL, 1), X = dd_fields(d, "sX", P_F64, BRIDGE_FULL, 1),
       RF = dd_fields(d, "sR", P_F64, BRIDGE_FULL, 1), TO = dd_fields(d, "sTo", P_F64, BRIDGE_ODD, 1);
  auto bh = dd_fields(d, "sbh", P_F64, BRIDGE_EVEN, 1), r = dd_fields(d, "sr", P_F64, BRIDGE_EVEN, 1),
       rh = dd_fields(d, "srh", P_F64, BRIDGE_EVEN, 1), pp = dd_fields(d, "sp", P_F64, BRIDGE_EVEN, 1),
       v = dd_fields(d, "sv", P_F64, BRIDGE_EVEN, 1), sv = dd_fields(d, "ss", P_F64, BRIDGE_EVEN, 1),
       t = dd_fields(d, "st", P_F64, BRIDGE_EVEN, 1), xe = dd_fields(d, "sxe", P_F64, BRIDGE_EVEN, 1);
  const Vec vB0{&B, 0}, vB1{&B, 1}, vX0{&X, 0}, vR0{&RF, 0}, vR1{&RF, 1};
  const Vec vbh{&bh, 0}, vr{&r, 0}, vrh{&rh, 0}, vp_{&pp, 0}, vv{&v, 0}, vs{&sv, 0}, vt{&t, 0}, vx{&xe, 0};
  const cx<double> one{1, 0}, zero{0, 0};
  for (int k = 0; k < nrhs; ++k) {
    bridge_info& inf = info[k];
    std::memset(&inf, 0, sizeof(inf));
    dd_fork(d);
    // b of this right-hand side into the slabs (its canonical slice has the global stride)
    for (int q = 0; q < d->nparts; ++q) {
      auto& s = d->slabs[q];
      canon_to_field(s.L, b_dev + ((long)k * V + (long)s.t0 * d->vs) * 24, B[q], s.L->stream, nullptr, V * 24);
    }
    // b^_e = T_ee^-1 (b_e + kappa H_eo T_oo^-1 b_o)
    for (int q = 0; q < d->nparts; ++q) {
      auto& s = d->slabs[q];
      if (clov)
        clover_site(s.L, P_F64, true, op_kcsw(d->op), 1, B[q], 1, TO[q], 1, 1, s.L->stream);
      else
        convert_field(s.L, B[q], TO[q], 1, s.L->stream, nullptr);
    }
    dd_prep(d, 0, bh, TO, B);
    cx<double> tmp;
    double b2 = 0, r2 = 0;
    dots(d, vbh, vbh, tmp, b2);
    lincomb(d, vx, {});
    lincomb(d, vr, {{one, vbh}});
    lincomb(d, vrh, {{one, vbh}});
    lincomb(d, vp_, {{one, vbh}});
    cx<double> rho{b2, 0}, alpha{1, 0}, omega{1, 0};
    const double tol2 = 0.01 * prm->tol * prm->tol * b2;
    int it = 0;
    r2 = b2;
    while (r2 > tol2 && it < max_iter && b2 > 0) {
      dd_dhat(d, P_F64, v, pp, TO);
      cx<double> rv;
      double vv2;
      dots(d, vrh, vv, rv, vv2);
      if (!(rv.r * rv.r + rv.i * rv.i > 0)) {
        inf.restarts += 1;
        break;
      }
      alpha = zdivd(rho, rv);
      lincomb(d, vs, {{one, vr}, {cx<double>{-alpha.r, -alpha.i}, vv}});
      dd_dhat(d, P_F64, t, sv, TO);
      // omega = <t, s> / |t|^2: dots(a, b) gives <a, b> and |b|^2, so take <s, t> and conjugate
      cx<double> st;
      double tt;
      dots(d, vs, vt, st, tt);
      omega = tt > 0 ? cx<double>{st.r / tt, -st.i / tt} : zero;
      lincomb(d, vx, {{one, vx}, {alpha, vp_}, {omega, vs}});
      lincomb(d, vr, {{one, vs}, {cx<double>{-omega.r, -omega.i}, vt}});
      cx<double> rho_new;
      dots(d, vrh, vr, rho_new, r2);
      ++it;
      if (r2 <= tol2) break;
      if (!(omega.r != 0 || omega.i != 0)) {
        inf.restarts += 1;
        break;
      }
      const cx<double> beta = zdivd(rho_new, rho) * zdivd(alpha, omega);
      const cx<double> bo = beta * omega;
      lincomb(d, vp_, {{one, vr}, {beta, vp_}, {cx<double>{-bo.r, -bo.i}, vv}});
      rho = rho_new;
    }
    // x_e, then x_o = T_oo^-1 (b_o + kappa H_oe x_e), then r = b - D x over the whole lattice
    lincomb(d, vX0, {{one, vx}});
    dd_prep(d, 1, X, X, B);
    dd_d(d, P_F64, RF, X);
    lincomb(d, vR0, {{one, vB0}, {cx<double>{-1, 0}, vR0}});
    lincomb(d, vR1, {{one, vB1}, {cx<double>{-1, 0}, vR1}});
    double n0, n1, bb0, bb1;
    dots(d, vR0, vR0, tmp, n0);
    dots(d, vR1, vR1, tmp, n1);
    dots(d, vB0, vB0, tmp, bb0);
    dots(d, vB1, vB1, tmp, bb1);
    for (int q = 0; q < d->nparts; ++q) {
      auto& s = d->slabs[q];
      field_to_canon(s.L, X[q], x_dev + ((long)k * V + (long)s.t0 * d->vs) * 24, s.L->stream, V * 24);
    }
    dd_join(d);
    BR_CUDA(cudaStreamSynchronize(d->global->stream));
    const double bn = bb0 + bb1;
    inf.true_rel_residual = bn > 0 ? std::sqrt((n0 + n1) / bn) : std::sqrt(n0 + n1);
    inf.inner_iters = it;
    inf.outer_iters = 1;
    inf.status = (bn == 0 || inf.true_rel_residual <= prm->tol) ? BRIDGE_OK
                 : std::isfinite(inf.true_rel_residual) ? BRIDGE_ENOCONV
                                                        : BRIDGE_EBREAKDOWN;
    inf.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  DD_END
}
