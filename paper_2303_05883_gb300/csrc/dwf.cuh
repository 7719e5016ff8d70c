// Moebius domain-wall kernels: the four-dimensional hopping term applied to
// every fifth-dimension slice, with the site-local fifth-dimension matrices
// fused into the epilogue.
//
// Operator (Sec. 2 of the paper implements Moebius domain-wall fermions and
// their even-odd blocks, Eq. 1, keeping the fifth coordinate s as an inner
// index of each four-dimensional site; the formula is the standard Moebius
// one):
//   D psi = (b W + 1) psi + (c W - 1) P psi,   W = (4 - M5) - H / 2,
//   (P psi)_s = P_- psi_{s+1} + P_+ psi_{s-1}   (wraps carry -m_f),
// so that, with the site-local A = (b(4-M5) + 1) + (c(4-M5) - 1) P and
// B = b + c P, D_ee = D_oo = A and D_eo, D_oe = -(1/2) H B.  Every
// site-local map is block diagonal in chirality (spins 0, 1: P_+; spins 2, 3:
// P_-) and acts on s through a real Ls x Ls matrix, the same at every site.
//
// A block of threads holds ns four-dimensional sites times all Ls slices
// (thread t: site t % ns, slice t / ns; the block is rounded up to whole
// warps, and threads past ns * Ls only join the barriers and reductions).  Each thread computes the hopping
// term of its (site, slice) with spin projection, exactly as the Wilson
// stencil does, and leaves it in shared memory; after one barrier each
// thread forms its output slice as a row of the s-matrix times the Ls hop
// results of its site.  The eight links of each site (row 2 rebuilt) and its
// neighbour indices are staged in shared memory once per block and read by
// all Ls slices of the site.
//
//   out_s = sum_t M1[s][t] (scale * H in)_t          (or scale * H in)
//         + s2 * self_s | sum_t M2[s][t] self_t      (optional)
//         + caux * aux_s                             (optional, aux != null)
//
// Epilogues: none, |out|^2 per right-hand side into a fused reduction, or
// the CG update x += alpha p, r -= alpha out with |r|^2 (out not stored).
#pragma once

#include "dslash.cuh"

namespace bridge {

enum DwfM2 { DM2_NONE = 0, DM2_PLAIN = 1, DM2_DENSE = 2 };
enum DwfEpi { DE_NONE = 0, DE_NORM = 1, DE_CGUPD = 2 };
enum DwfMixMode { DX_PLAIN = 0, DX_CGP = 1 };

// A fifth-dimension matrix as a product of at most two cyclic bidiagonal
// factors per chirality, applied right to left, then a sign:
//   MUL   y_s = d x_s + e x_{s+dir}          (x_{Ls} -> -m_f x_0, x_{-1} -> -m_f x_{Ls-1})
//   SOLVE d y_s + e y_{s+dir} = x_s          (the same cyclic system, solved)
// A = d + e S and B = b + c S are of this form with dir = -1 on the P_+
// components and +1 on the P_- ones (S the s-part of P); transposes flip
// dir.  SOLVE runs a first-order recurrence in the direction that damps
// (|e/d| <= 1, checked on the host; otherwise the dense matrix is used).
enum SFacKind { SF_MUL = 0, SF_SOLVE = 1 };
struct SProg {
  int nf[2];  // factors per chirality (0 = identity)
  int kind[2][2], dir[2][2];
  double d[2][2], e[2][2];
  double sign[2];
};

// In-place factors on one column x_0 .. x_{Ls-1} of a site's staged values
// (elements `stride` apart in shared memory).
template <class R>
BR_D void col_mul(cx<R>* col, int stride, int Ls, R d, R e, int dir, R mf) {
  if (dir < 0) {
    const cx<R> last = col[(long)(Ls - 1) * stride];
    for (int s = Ls - 1; s >= 1; --s) col[(long)s * stride] = d * col[(long)s * stride] + e * col[(long)(s - 1) * stride];
    col[0] = d * col[0] + (-mf * e) * last;
  } else {
    const cx<R> first = col[0];
    for (int s = 0; s < Ls - 1; ++s) col[(long)s * stride] = d * col[(long)s * stride] + e * col[(long)(s + 1) * stride];
    col[(long)(Ls - 1) * stride] = d * col[(long)(Ls - 1) * stride] + (-mf * e) * first;
  }
}

template <class R>
BR_D void col_solve(cx<R>* col, int stride, int Ls, R d, R e, int dir, R mf) {
  // With r = -e/d: the end value follows from the wrap equation in closed
  // form, the rest from y = x/d + r y(previous) along dir.
  const R r = -e / d, inv_d = R(1) / d;
  cx<R> acc = czero<R>();
  R w = R(1);
  if (dir < 0) {
    for (int t = Ls - 1; t >= 1; --t) {
      acc = acc + w * col[(long)t * stride];
      w *= r;
    }
    cx<R> y = (R(1) / (d - e * mf * w)) * (col[0] + (e * mf * inv_d) * acc);
    col[0] = y;
    for (int s = 1; s < Ls; ++s) {
      y = inv_d * col[(long)s * stride] + r * y;
      col[(long)s * stride] = y;
    }
  } else {
    for (int t = 0; t <= Ls - 2; ++t) {
      acc = acc + w * col[(long)t * stride];
      w *= r;
    }
    cx<R> y = (R(1) / (d - e * mf * w)) * (col[(long)(Ls - 1) * stride] + (e * mf * inv_d) * acc);
    col[(long)(Ls - 1) * stride] = y;
    for (int s = Ls - 2; s >= 0; --s) {
      y = inv_d * col[(long)s * stride] + r * y;
      col[(long)s * stride] = y;
    }
  }
}

// Apply a program to every (site, component) column of sh[Ls][12][ns];
// must be reached by every thread of the block (it ends with a barrier).
template <class R>
BR_D void prog_columns(const SProg& pg, cx<R>* sh, int Ls, int ns, R mf) {
  for (int cidx = threadIdx.x; cidx < 12 * ns; cidx += blockDim.x) {
    const int sl = cidx % ns, k = cidx / ns, chi = k < 6 ? 0 : 1;
    cx<R>* col = sh + (long)k * ns + sl;
    const int stride = 12 * ns;
    for (int f = 0; f < pg.nf[chi]; ++f) {
      if (pg.kind[chi][f] == SF_MUL)
        col_mul<R>(col, stride, Ls, (R)pg.d[chi][f], (R)pg.e[chi][f], pg.dir[chi][f], mf);
      else
        col_solve<R>(col, stride, Ls, (R)pg.d[chi][f], (R)pg.e[chi][f], pg.dir[chi][f], mf);
    }
    const R sg = (R)pg.sign[chi];
    if (sg != R(1))
      for (int t = 0; t < Ls; ++t) col[(long)t * stride] = sg * col[(long)t * stride];
  }
  __syncthreads();
}

// The same programs with a whole column in registers (FP32, compile-time
// Ls): one shared-memory load and one store per element instead of a load,
// a dependent FMA and a store per step of each factor, so the sweep is no
// longer a chain of shared-memory round trips.  Same operations in the same
// order as col_mul / col_solve.
template <class R, int LS>
BR_D void col_mul_reg(cx<R> v[LS], R d, R e, int dir, R mf) {
  if (dir < 0) {
    const cx<R> last = v[LS - 1];
#pragma unroll
    for (int s = LS - 1; s >= 1; --s) v[s] = d * v[s] + e * v[s - 1];
    v[0] = d * v[0] + (-mf * e) * last;
  } else {
    const cx<R> first = v[0];
#pragma unroll
    for (int s = 0; s < LS - 1; ++s) v[s] = d * v[s] + e * v[s + 1];
    v[LS - 1] = d * v[LS - 1] + (-mf * e) * first;
  }
}

template <class R, int LS>
BR_D void col_solve_reg(cx<R> v[LS], R d, R e, int dir, R mf) {
  const R r = -e / d, inv_d = R(1) / d;
  cx<R> acc = czero<R>();
  R w = R(1);
  if (dir < 0) {
#pragma unroll
    for (int t = LS - 1; t >= 1; --t) {
      acc = acc + w * v[t];
      w *= r;
    }
    cx<R> y = (R(1) / (d - e * mf * w)) * (v[0] + (e * mf * inv_d) * acc);
    v[0] = y;
#pragma unroll
    for (int s = 1; s < LS; ++s) {
      y = inv_d * v[s] + r * y;
      v[s] = y;
    }
  } else {
#pragma unroll
    for (int t = 0; t <= LS - 2; ++t) {
      acc = acc + w * v[t];
      w *= r;
    }
    cx<R> y = (R(1) / (d - e * mf * w)) * (v[LS - 1] + (e * mf * inv_d) * acc);
    v[LS - 1] = y;
#pragma unroll
    for (int s = LS - 2; s >= 0; --s) {
      y = inv_d * v[s] + r * y;
      v[s] = y;
    }
  }
}

template <class R, int LS>
BR_D void prog_columns_reg(const SProg& pg, cx<R>* sh, int ns, R mf) {
  for (int cidx = threadIdx.x; cidx < 12 * ns; cidx += blockDim.x) {
    const int sl = cidx % ns, k = cidx / ns, chi = k < 6 ? 0 : 1;
    cx<R>* col = sh + (long)k * ns + sl;
    const long stride = 12L * ns;
    cx<R> v[LS];
#pragma unroll
    for (int s = 0; s < LS; ++s) v[s] = col[s * stride];
    for (int f = 0; f < pg.nf[chi]; ++f) {
      if (pg.kind[chi][f] == SF_MUL)
        col_mul_reg<R, LS>(v, (R)pg.d[chi][f], (R)pg.e[chi][f], pg.dir[chi][f], mf);
      else
        col_solve_reg<R, LS>(v, (R)pg.d[chi][f], (R)pg.e[chi][f], pg.dir[chi][f], mf);
    }
    const R sg = (R)pg.sign[chi];
#pragma unroll
    for (int s = 0; s < LS; ++s) col[s * stride] = sg != R(1) ? sg * v[s] : v[s];
  }
  __syncthreads();
}

// The register form for FP32 and the usual Ls, else the shared-memory one.
template <class R>
BR_D void prog_columns_any(const SProg& pg, cx<R>* sh, int Ls, int ns, R mf) {
  if constexpr (sizeof(R) == 4) {
    if (Ls == 16) {
      prog_columns_reg<R, 16>(pg, sh, ns, mf);
      return;
    }
    if (Ls == 8) {
      prog_columns_reg<R, 8>(pg, sh, ns, mf);
      return;
    }
  }
  prog_columns<R>(pg, sh, Ls, ns, mf);
}

struct DwfArgs {
  Geom g;
  int out_parity;
  int Ls, nrhs;
  int ns;   // four-dimensional sites per block (blockDim = ns * Ls rounded up to 32, <= 256)
  int nsb;  // site blocks per right-hand side (grid = nsb * nrhs)
  double scale, s2, caux;
  float scalef, s2f, cauxf;
  double bc[4];
  float bcf[4];
  // bytes between consecutive slices (slice q = rhs * Ls + s) of each operand;
  // x, r and p of the CG update share cg_bs
  long in_bs, out_bs, self_bs, aux_bs, cg_bs;
  char* out;
  const char* in;
  const char* self;
  const char* aux;
  char* x;  // CG update epilogue
  char* r;
  const char* p;
  const char* gauge;  // [parity][mu] link blocks
  const void* m1;     // [2][Ls][Ls] in the compute precision (chirality +, then -)
  const void* m2;
  int fact;           // 1: apply m1 / m2 by their bidiagonal factors p1 / p2 (no dense matrices staged)
  double mf;
  SProg p1, p2;
  RedArgs red;
};

struct DwfMixArgs {
  uint32_t vh;
  int Ls, nrhs, ns, nsb;
  long in_bs, out_bs, cg_bs;  // slice strides (cg_bs for p and r)
  char* out;        // out = M in (DX_PLAIN) or M p (DX_CGP)
  const char* in;
  char* p;          // DX_CGP: p = r + beta p, stored
  const char* r;
  const void* m;
  RedArgs red;      // DX_CGP: beta and done flags from red.cg
  double s0;        // DX_PLAIN: out = s0 * in + M in when s0 != 0
  float s0f;
  int fact;         // 1: apply m by its bidiagonal factors pm
  double mf;
  SProg pm;
};

BR_HD int dwf_threads(int ns, int Ls) { return (ns * Ls + 31) / 32 * 32; }

// Dynamic shared memory of one block: the s-matrices and ns * Ls spinors
// per staged operand.
BR_HD long dwf_hop_smem(int prec, int Ls, int ns, bool m1, bool m2dense, bool fact) {
  const long R = prec == P_F64 ? 8 : 4;
  const long mats = fact ? 0 : (m1 ? 1 : 0) + (m2dense ? 1 : 0);
  const long vecs = (m1 ? 1 : 0) + (m2dense ? 1 : 0);
  const long links = 8L * 9 * ns * 2 * R + 8L * ns * 4;  // staged links and neighbour words
  return links + mats * 2 * Ls * Ls * R + vecs * (long)Ls * 12 * ns * 2 * R;
}
BR_HD long dwf_mix_smem(int prec, int Ls, int ns, bool fact) {
  const long R = prec == P_F64 ? 8 : 4;
  return (fact ? 0 : 2L * Ls * Ls * R) + (long)Ls * 12 * ns * 2 * R;
}

// Row s of the chirality-blocked s-matrix applied to the Ls staged spinors
// of one site: res[k] = sum_t M[chi(k)][s][t] sh[t][k].
template <class R>
BR_D void smix_row(const R* mat, const cx<R>* sh, int Ls, int ns, int s, int sl, cx<R> res[12]) {
#pragma unroll
  for (int k = 0; k < 12; ++k) res[k] = czero<R>();
  const R* rp = mat + (long)s * Ls;            // chirality + (spins 0, 1)
  const R* rm = mat + (long)(Ls + s) * Ls;     // chirality - (spins 2, 3)
  for (int t = 0; t < Ls; ++t) {
    const R a = rp[t], b = rm[t];
    const cx<R>* v = sh + (long)t * 12 * ns + sl;
#pragma unroll
    for (int k = 0; k < 6; ++k) res[k] = caxpy(a, v[k * ns], res[k]);
#pragma unroll
    for (int k = 6; k < 12; ++k) res[k] = caxpy(b, v[k * ns], res[k]);
  }
}

template <class R>
BR_D void stage_row(cx<R>* sh, int ns, int s, int sl, const cx<R> v[12]) {
#pragma unroll
  for (int k = 0; k < 12; ++k) sh[((long)s * 12 + k) * ns + sl] = v[k];
}

// One hop from shared data: the link (9 complex entries, stride ns) and the
// neighbour index with its wrap flag in bit 31, staged once per site.
template <int P, int MU, bool FWD>
BR_D void hop_shared(const char* in, long vh, uint32_t nbw, const cx<typename Tr<P>::R>* lk, int ns,
                     typename Tr<P>::R bc, cx<typename Tr<P>::R> acc[12]) {
  using R = typename Tr<P>::R;
  const uint32_t nb = nbw & 0x7fffffffu;
  cx<R> h[2][3];
  {
    cx<R> psi[12];
    load_spinor<P>(in, vh, nb, psi);
    project<R, MU, FWD>(psi, h);
  }
  if (nbw >> 31) {
#pragma unroll
    for (int k = 0; k < 2; ++k)
#pragma unroll
      for (int c = 0; c < 3; ++c) h[k][c] = bc * h[k][c];
  }
  cx<R> U[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) U[k] = lk[k * ns];
  cx<R> u[2][3];
#pragma unroll
  for (int k = 0; k < 2; ++k)
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      if (FWD)
        u[k][r] = crow3(U[3 * r], U[3 * r + 1], U[3 * r + 2], h[k]);
      else
        u[k][r] = crow3_conj(U[r], U[3 + r], U[6 + r], h[k]);
    }
  reconstruct<R, MU, FWD>(u, acc);
}

// The same hop for SPT slices of one site (slices q0 + j * qstep): the link,
// the neighbour index and its address arithmetic are read once and shared.
template <int P, int MU, bool FWD, int SPT>
BR_D void hop_shared_multi(const char* in, long in_bs, long qstep, long vh, uint32_t nbw,
                           const cx<typename Tr<P>::R>* lk, int ns, typename Tr<P>::R bc,
                           cx<typename Tr<P>::R> acc[SPT][12]) {
  using R = typename Tr<P>::R;
  const uint32_t nb = nbw & 0x7fffffffu;
  const bool wraps = (nbw >> 31) != 0;
  cx<R> U[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) U[k] = lk[k * ns];
#pragma unroll
  for (int j = 0; j < SPT; ++j) {
    cx<R> h[2][3];
    {
      cx<R> psi[12];
      load_spinor<P>(in + j * qstep * in_bs, vh, nb, psi);
      project<R, MU, FWD>(psi, h);
    }
    if (wraps) {
#pragma unroll
      for (int k = 0; k < 2; ++k)
#pragma unroll
        for (int c = 0; c < 3; ++c) h[k][c] = bc * h[k][c];
    }
    cx<R> u[2][3];
#pragma unroll
    for (int k = 0; k < 2; ++k)
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        if (FWD)
          u[k][r] = crow3(U[3 * r], U[3 * r + 1], U[3 * r + 2], h[k]);
        else
          u[k][r] = crow3_conj(U[r], U[3 + r], U[6 + r], h[k]);
      }
    reconstruct<R, MU, FWD>(u, acc[j]);
  }
}

// Stage the links and neighbour indices of the block's ns sites: entry
// d = 2 mu + (0 forward, 1 backward) holds U_mu(x) or U_mu(x - mu) with all 9
// entries (row 2 rebuilt for 12-real storage) at shl[(d * 9 + k) * ns + site].
template <int P>
BR_D void stage_links(const DwfArgs& a, int sb, cx<typename Tr<P>::R>* shl, uint32_t* shn) {
  using R = typename Tr<P>::R;
  const int ns = a.ns, p = a.out_parity;
  const long vh = a.g.vh;
  const long lbb = link_block_bytes(P, vh);
  const char* g_out = a.gauge + (long)p * 4 * lbb;
  const char* g_in = a.gauge + (long)(1 - p) * 4 * lbb;
  for (int i = threadIdx.x; i < 8 * ns; i += blockDim.x) {
    const int sl = i % ns, d = i / ns, mu = d >> 1;
    const bool fwd = (d & 1) == 0;
    const uint32_t ih = (uint32_t)sb * ns + sl;
    if (ih >= (uint32_t)vh) continue;
    int c[4];
    uint32_t xh, f, b;
    bool wf, wb;
    site_coords(a.g, ih, p, c, xh);
    switch (mu) {
      case 0: neighbours<0>(a.g, ih, c, xh, f, b, wf, wb); break;
      case 1: neighbours<1>(a.g, ih, c, xh, f, b, wf, wb); break;
      case 2: neighbours<2>(a.g, ih, c, xh, f, b, wf, wb); break;
      default: neighbours<3>(a.g, ih, c, xh, f, b, wf, wb); break;
    }
    Link<R> U;
    load_link<P, true>((fwd ? g_out : g_in) + mu * lbb, vh, fwd ? ih : b, U);
#pragma unroll
    for (int k = 0; k < 9; ++k) shl[((long)d * 9 + k) * ns + sl] = U.m[k / 3][k % 3];
    shn[d * ns + sl] = (fwd ? f : b) | ((fwd ? wf : wb) ? 0x80000000u : 0u);
  }
}

// MINB: resident 256-thread blocks per SM the register allocation must allow
// (1: no cap, 2: <= 128 registers, 3: <= 85, 4: <= 64); SPT: slices per
// thread (1, or 2 for even Ls: slices s and s + Ls / 2 of one site share the
// link reads, neighbour index and address arithmetic of every hop, and give
// the thread two independent FMA chains).  Picked per kernel by the tuner.
template <int P, bool M1, int M2, int EPI, int MINB = 2, int SPT = 1>
__global__ void __launch_bounds__(256, MINB) dwf_hop_kernel(const DwfArgs a) {
  using R = typename Tr<P>::R;
  extern __shared__ __align__(16) unsigned char dsm[];
  const int Ls = a.Ls, ns = a.ns;
  const int nm = 2 * Ls * Ls;
  const int lss = Ls / SPT;  // slice groups
  cx<R>* shl = reinterpret_cast<cx<R>*>(dsm);                 // [8][9][ns] links
  uint32_t* shn = reinterpret_cast<uint32_t*>(shl + 72L * ns);  // [8][ns] neighbours
  const bool fact = a.fact != 0;
  R* mat1 = reinterpret_cast<R*>(shn + 8L * ns);
  R* mat2 = mat1 + ((M1 && !fact) ? nm : 0);
  cx<R>* shh = reinterpret_cast<cx<R>*>(mat2 + ((M2 == DM2_DENSE && !fact) ? nm : 0));
  cx<R>* shs = shh + (M1 ? (long)Ls * 12 * ns : 0);

  const int rhs = blockIdx.x % a.nrhs;
  const int sb = blockIdx.x / a.nrhs;
  // site and slice group of this thread: with two slices per thread a warp
  // takes 16 sites x 2 slice groups (when the block's shape allows), so that
  // each 8-byte link read from shared memory touches 16 sites -- one
  // 128-byte wavefront -- while serving four slices of each; otherwise
  // consecutive threads take consecutive sites
  int sl = threadIdx.x % ns, s0 = threadIdx.x / ns;
  if (SPT == 2 && ns % 16 == 0 && lss % 2 == 0 && ns * lss == (int)blockDim.x) {
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, nst = ns / 16;
    sl = 16 * (w % nst) + (lane & 15);
    s0 = 2 * (w / nst) + (lane >> 4);
  }
  const uint32_t ih = (uint32_t)sb * ns + sl;
  const long vh = a.g.vh;
  const bool live = s0 < lss;
  const bool skip = a.red.check_done && a.red.cg != nullptr && a.red.cg[rhs].done != RUNNING;
  const bool valid = live && ih < (uint32_t)vh && !skip;
  const long q0 = (long)rhs * Ls + s0;  // slice j of this thread: q0 + j * lss

  if (M1 && !fact)
    for (int i = threadIdx.x; i < nm; i += blockDim.x) mat1[i] = reinterpret_cast<const R*>(a.m1)[i];
  if (M2 == DM2_DENSE && !fact)
    for (int i = threadIdx.x; i < nm; i += blockDim.x) mat2[i] = reinterpret_cast<const R*>(a.m2)[i];
  if (!skip) stage_links<P>(a, sb, shl, shn);
  __syncthreads();

  cx<R> acc[SPT][12];
#pragma unroll
  for (int j = 0; j < SPT; ++j)
#pragma unroll
    for (int k = 0; k < 12; ++k) acc[j][k] = czero<R>();
  if (valid) {
    const char* in = a.in + q0 * a.in_bs;
    const cx<R>* lk = shl + sl;
    const uint32_t* nw = shn + sl;
    hop_shared_multi<P, 0, true, SPT>(in, a.in_bs, lss, vh, nw[0 * ns], lk + 0 * 9 * ns, ns, pick<R>(a.bc[0], a.bcf[0]), acc);
    hop_shared_multi<P, 0, false, SPT>(in, a.in_bs, lss, vh, nw[1 * ns], lk + 1 * 9 * ns, ns, pick<R>(a.bc[0], a.bcf[0]), acc);
    hop_shared_multi<P, 1, true, SPT>(in, a.in_bs, lss, vh, nw[2 * ns], lk + 2 * 9 * ns, ns, pick<R>(a.bc[1], a.bcf[1]), acc);
    hop_shared_multi<P, 1, false, SPT>(in, a.in_bs, lss, vh, nw[3 * ns], lk + 3 * 9 * ns, ns, pick<R>(a.bc[1], a.bcf[1]), acc);
    hop_shared_multi<P, 2, true, SPT>(in, a.in_bs, lss, vh, nw[4 * ns], lk + 4 * 9 * ns, ns, pick<R>(a.bc[2], a.bcf[2]), acc);
    hop_shared_multi<P, 2, false, SPT>(in, a.in_bs, lss, vh, nw[5 * ns], lk + 5 * 9 * ns, ns, pick<R>(a.bc[2], a.bcf[2]), acc);
    hop_shared_multi<P, 3, true, SPT>(in, a.in_bs, lss, vh, nw[6 * ns], lk + 6 * 9 * ns, ns, pick<R>(a.bc[3], a.bcf[3]), acc);
    hop_shared_multi<P, 3, false, SPT>(in, a.in_bs, lss, vh, nw[7 * ns], lk + 7 * 9 * ns, ns, pick<R>(a.bc[3], a.bcf[3]), acc);
    const R sc = pick<R>(a.scale, a.scalef);
#pragma unroll
    for (int j = 0; j < SPT; ++j)
#pragma unroll
      for (int k = 0; k < 12; ++k) acc[j][k] = sc * acc[j][k];
  }
  if (M1 && live)
#pragma unroll
    for (int j = 0; j < SPT; ++j) stage_row(shh, ns, s0 + j * lss, sl, acc[j]);
  if (M2 == DM2_DENSE && live) {
#pragma unroll
    for (int j = 0; j < SPT; ++j) {
      cx<R> v[12];
      if (valid) {
        load_spinor<P>(a.self + (q0 + j * lss) * a.self_bs, vh, ih, v);
      } else {
#pragma unroll
        for (int k = 0; k < 12; ++k) v[k] = czero<R>();
      }
      stage_row(shs, ns, s0 + j * lss, sl, v);
    }
  }
  if (M1 || M2 == DM2_DENSE) __syncthreads();
  if (fact) {
    if (M1) prog_columns_any<R>(a.p1, shh, Ls, ns, (R)a.mf);
    if (M2 == DM2_DENSE) prog_columns_any<R>(a.p2, shs, Ls, ns, (R)a.mf);
  }

  R nrm = R(0);
  if (valid) {
#pragma unroll
    for (int j = 0; j < SPT; ++j) {
      const int s = s0 + j * lss;
      const long q = q0 + (long)j * lss;
      cx<R> v[12];
      if (M1 && fact) {
#pragma unroll
        for (int k = 0; k < 12; ++k) v[k] = shh[((long)s * 12 + k) * ns + sl];
      } else if (M1) {
        smix_row(mat1, shh, Ls, ns, s, sl, v);
      } else {
#pragma unroll
        for (int k = 0; k < 12; ++k) v[k] = acc[j][k];
      }
      if (M2 == DM2_PLAIN) {
        cx<R> w[12];
        load_spinor<P>(a.self + q * a.self_bs, vh, ih, w);
        const R s2 = pick<R>(a.s2, a.s2f);
#pragma unroll
        for (int k = 0; k < 12; ++k) v[k] = v[k] + s2 * w[k];
      } else if (M2 == DM2_DENSE) {
        cx<R> w[12];
        if (fact) {
#pragma unroll
          for (int k = 0; k < 12; ++k) w[k] = shs[((long)s * 12 + k) * ns + sl];
        } else {
          smix_row(mat2, shs, Ls, ns, s, sl, w);
        }
#pragma unroll
        for (int k = 0; k < 12; ++k) v[k] = v[k] + w[k];
      }
      if (a.aux != nullptr) {
        cx<R> w[12];
        load_spinor<P>(a.aux + q * a.aux_bs, vh, ih, w);
        const R ca = pick<R>(a.caux, a.cauxf);
#pragma unroll
        for (int k = 0; k < 12; ++k) v[k] = v[k] + ca * w[k];
      }
      if (EPI == DE_CGUPD) {
        const R alpha = (R)a.red.cg[rhs].alpha;
        cx<R> xv[12], rv[12], pv[12];
        load_spinor<P, false>(a.x + q * a.cg_bs, vh, ih, xv);
        load_spinor<P, false>(a.r + q * a.cg_bs, vh, ih, rv);
        load_spinor<P>(a.p + q * a.cg_bs, vh, ih, pv);
#pragma unroll
        for (int k = 0; k < 12; ++k) {
          xv[k] = xv[k] + alpha * pv[k];
          rv[k] = rv[k] - alpha * v[k];
          nrm += rv[k].r * rv[k].r + rv[k].i * rv[k].i;
        }
        store_spinor<P>(a.x + q * a.cg_bs, vh, ih, xv);
        store_spinor<P>(a.r + q * a.cg_bs, vh, ih, rv);
      } else {
        store_spinor<P>(a.out + q * a.out_bs, vh, ih, v);
        if (EPI == DE_NORM)
#pragma unroll
          for (int k = 0; k < 12; ++k) nrm += v[k].r * v[k].r + v[k].i * v[k].i;
      }
    }
  }
  if (EPI != DE_NONE) {
    double rv[1] = {(double)nrm};
    reduce_finalize<1>(a.red, rhs, sb, a.nsb, a.nrhs, rv);
  }
}

// out = M in per site (DX_PLAIN, optionally + s0 in), or the CG direction
// update p = r + beta p followed by out = M p (DX_CGP).
template <int P, int MODE, int MINB = 2>
__global__ void __launch_bounds__(256, MINB) dwf_mix_kernel(const DwfMixArgs a) {
  using R = typename Tr<P>::R;
  extern __shared__ __align__(16) unsigned char dsm[];
  const int Ls = a.Ls, ns = a.ns;
  const int nm = 2 * Ls * Ls;
  const bool fact = a.fact != 0;
  R* mat = reinterpret_cast<R*>(dsm);
  cx<R>* sh = reinterpret_cast<cx<R>*>(mat + (fact ? 0 : nm));
  const int rhs = blockIdx.x % a.nrhs;
  const int sb = blockIdx.x / a.nrhs;
  const int sl = threadIdx.x % ns, s = threadIdx.x / ns;
  const uint32_t ih = (uint32_t)sb * ns + sl;
  const bool live = s < Ls;
  const bool skip = MODE == DX_CGP && a.red.cg != nullptr && a.red.cg[rhs].done != RUNNING;
  const bool valid = live && ih < a.vh && !skip;
  const long q = (long)rhs * Ls + s;
  if (!fact)
    for (int i = threadIdx.x; i < nm; i += blockDim.x) mat[i] = reinterpret_cast<const R*>(a.m)[i];
  cx<R> v[12];
  if (valid) {
    if (MODE == DX_CGP) {
      const R beta = (R)a.red.cg[rhs].beta;
      cx<R> rv[12];
      load_spinor<P>(a.r + q * a.cg_bs, a.vh, ih, rv);
      load_spinor<P, false>(a.p + q * a.cg_bs, a.vh, ih, v);
#pragma unroll
      for (int k = 0; k < 12; ++k) v[k] = rv[k] + beta * v[k];
      store_spinor<P>(a.p + q * a.cg_bs, a.vh, ih, v);
    } else {
      load_spinor<P>(a.in + q * a.in_bs, a.vh, ih, v);
    }
  } else {
#pragma unroll
    for (int k = 0; k < 12; ++k) v[k] = czero<R>();
  }
  if (live) stage_row(sh, ns, s, sl, v);
  __syncthreads();
  if (fact) prog_columns_any<R>(a.pm, sh, Ls, ns, (R)a.mf);
  if (valid) {
    cx<R> w[12];
    if (fact) {
#pragma unroll
      for (int k = 0; k < 12; ++k) w[k] = sh[((long)s * 12 + k) * ns + sl];
    } else {
      smix_row(mat, sh, Ls, ns, s, sl, w);
    }
    if (MODE == DX_PLAIN && a.s0 != 0.0) {
      const R s0 = pick<R>(a.s0, a.s0f);
#pragma unroll
      for (int k = 0; k < 12; ++k) w[k] = w[k] + s0 * v[k];
    }
    store_spinor<P>(a.out + q * a.out_bs, a.vh, ih, w);
  }
}

}  // namespace bridge
