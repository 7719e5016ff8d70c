// The Wilson/clover hopping stencil and its fused epilogues.
//
// Operator (Sec. 2 of the paper implements the Wilson and clover fermion
// operators and their even-odd blocks, Eq. 1; the formula is the standard
// one, with the chiral gamma basis):
//   (H psi)(x) = sum_mu (1 - gamma_mu) U_mu(x) psi(x+mu)
//              + (1 + gamma_mu) U_mu(x-mu)^dagger psi(x-mu),
// boundary phase bc[mu] on every hop that wraps around the lattice.
//
// One thread computes one output site of one right-hand side.  Each of the
// eight hops projects the neighbour spinor onto its two independent spin
// components (a half spinor), multiplies by the link, and reconstructs the
// other two, so only 2 x (3x3 complex matrix times 3-vector) per hop.  The
// result of the hop term is combined in registers:
//
//   out = s1 * M(self) + E( beta * H(in) + caux * aux )
//
// with M in {1, T} (F_SELF, F_SELF_CLOV) and E in {1, T^-1, gamma5}
// (F_E_CLOV, F_G5: the second pass of the adjoint Schur operator); this
// single kernel covers D_eo / D_oe, the full operator T - kappa H, both
// passes of the Schur operator of Eq. 1, the even-odd source preparation and
// solution reconstruction, and the FP64 residual b - D x.  Optional fused
// reductions: |out|^2, <a, out>, or (<out, self>, |out|^2).
#pragma once

#include "common.cuh"
#include "reduce.cuh"

namespace bridge {

enum HopFlags { F_SELF = 1, F_SELF_CLOV = 2, F_E_CLOV = 4, F_AUX = 8, F_G5 = 16 };

// A right-hand side whose solve has ended (BiCGStab or CG scalars) is skipped.
BR_D bool rhs_finished(const RedArgs& r, int rhs) {
  return r.check_done && ((r.sc != nullptr && r.sc[rhs].done != RUNNING) || (r.cg != nullptr && r.cg[rhs].done != RUNNING));
}
enum RedMode { R_NONE = 0, R_NORM = 1, R_DOT_A = 2, R_TS = 3 };

struct HopArgs {
  Geom g;
  int out_parity;
  int nrhs;
  int nblk;  // site blocks per right-hand side (grid = nblk * nrhs)
  double beta, s1, caux;
  double bc[4];
  float betaf, s1f, cauxf, bcf[4];  // the same in FP32 for the FP32-math kernels
  // Field pointers address the block of the right parity for rhs 0; *_rs is
  // the byte stride between right-hand sides.
  char* out;
  long out_rs;
  const char* in;
  long in_rs;
  const char* self;
  long self_rs;
  const char* aux;
  long aux_rs;
  const char* avec;
  long avec_rs;
  const char* gauge;  // [parity][mu] link blocks
  const char* clovE;  // [parity] clover blocks (T^-1)
  const char* clovM;  // [parity] clover blocks (T)
  RedArgs red;
  // Non-null: compute only the n_map output sites site_map[0 .. n_map) (half-
  // lattice indices, ascending; e.g. the sites of one colour of a Schwarz
  // blocking); the other sites are neither read nor written.
  const uint32_t* site_map;
  uint32_t n_map;
};

template <class R, int MU, bool FWD>
BR_D void project(const cx<R> p[12], cx<R> h[2][3]) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const cx<R> p0 = p[c], p1 = p[3 + c], p2 = p[6 + c], p3 = p[9 + c];
    if (MU == 0) {
      h[0][c] = FWD ? p0 + times_i(p3) : p0 - times_i(p3);
      h[1][c] = FWD ? p1 + times_i(p2) : p1 - times_i(p2);
    } else if (MU == 1) {
      h[0][c] = FWD ? p0 + p3 : p0 - p3;
      h[1][c] = FWD ? p1 - p2 : p1 + p2;
    } else if (MU == 2) {
      h[0][c] = FWD ? p0 + times_i(p2) : p0 - times_i(p2);
      h[1][c] = FWD ? p1 - times_i(p3) : p1 + times_i(p3);
    } else {
      h[0][c] = FWD ? p0 - p2 : p0 + p2;
      h[1][c] = FWD ? p1 - p3 : p1 + p3;
    }
  }
}

template <class R, int MU, bool FWD>
BR_D void reconstruct(const cx<R> u[2][3], cx<R> acc[12]) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const cx<R> u0 = u[0][c], u1 = u[1][c];
    acc[c] = acc[c] + u0;
    acc[3 + c] = acc[3 + c] + u1;
    if (MU == 0) {
      acc[6 + c] = FWD ? acc[6 + c] + times_mi(u1) : acc[6 + c] + times_i(u1);
      acc[9 + c] = FWD ? acc[9 + c] + times_mi(u0) : acc[9 + c] + times_i(u0);
    } else if (MU == 1) {
      acc[6 + c] = FWD ? acc[6 + c] - u1 : acc[6 + c] + u1;
      acc[9 + c] = FWD ? acc[9 + c] + u0 : acc[9 + c] - u0;
    } else if (MU == 2) {
      acc[6 + c] = FWD ? acc[6 + c] + times_mi(u0) : acc[6 + c] + times_i(u0);
      acc[9 + c] = FWD ? acc[9 + c] + times_i(u1) : acc[9 + c] + times_mi(u1);
    } else {
      acc[6 + c] = FWD ? acc[6 + c] - u0 : acc[6 + c] + u0;
      acc[9 + c] = FWD ? acc[9 + c] - u1 : acc[9 + c] + u1;
    }
  }
}

// One hop: psi at half-lattice site nb of the input, link block lb at index li.
template <int P, int MU, bool FWD, bool ST>
BR_D void hop_one(const char* in, const char* lb, long vh, uint32_t nb, uint32_t li, bool wraps,
                  typename Tr<P>::R bc, cx<typename Tr<P>::R> acc[12]) {
  using R = typename Tr<P>::R;
  cx<R> h[2][3];
  if constexpr (Tr<P>::half) {
    // project the stored values, then apply the per-site scale and the
    // boundary phase to the 12 projected components only
    cx<float> psi[12];
    const float sc = load_spinor_unscaled<P>(in, vh, nb, psi) * (wraps ? bc : 1.0f);
    project<R, MU, FWD>(psi, h);
#pragma unroll
    for (int k = 0; k < 2; ++k)
#pragma unroll
      for (int c = 0; c < 3; ++c) h[k][c] = sc * h[k][c];
  } else {
    {
      cx<R> psi[12];
      load_spinor<P>(in, vh, nb, psi);
      project<R, MU, FWD>(psi, h);
    }
    if (wraps) {
#pragma unroll
      for (int k = 0; k < 2; ++k)
#pragma unroll
        for (int c = 0; c < 3; ++c) h[k][c] = bc * h[k][c];
    }
  }
  Link<R> U;
  load_link<P, ST>(lb, vh, li, U);
  cx<R> u[2][3];
#pragma unroll
  for (int k = 0; k < 2; ++k)
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      if (FWD)
        u[k][r] = crow3(U.m[r][0], U.m[r][1], U.m[r][2], h[k]);
      else
        u[k][r] = crow3_conj(U.m[0][r], U.m[1][r], U.m[2][r], h[k]);
    }
  reconstruct<R, MU, FWD>(u, acc);
}

template <class R>
BR_HD R pick(double d, float f) {
  if constexpr (sizeof(R) == sizeof(double)) {
    return d;
  } else {
    return f;
  }
}

template <int P, int MU, bool ST>
BR_D void hop_dir(const HopArgs& a, const char* in, const char* g_out, const char* g_in, long lbb, uint32_t ih,
                  const int c[4], uint32_t xh, cx<typename Tr<P>::R> acc[12]) {
  using R = typename Tr<P>::R;
  uint32_t f, b;
  bool wf, wb;
  neighbours<MU>(a.g, ih, c, xh, f, b, wf, wb);
  const R bc = pick<R>(a.bc[MU], a.bcf[MU]);
  // forward: link U_mu(x) lives at x (output parity); backward: U_mu(x - mu) at x - mu.
  hop_one<P, MU, true, ST>(in, g_out + MU * lbb, a.g.vh, f, ih, wf, bc, acc);
  hop_one<P, MU, false, ST>(in, g_in + MU * lbb, a.g.vh, b, b, wb, bc, acc);
}

// MINB: minimum resident 256-thread blocks per SM the compiler must allow
// (1 = no register cap, 3 = <= 80 registers, 4 = <= 64 registers); ST:
// load the read-once operands around L1 (see ldg4).  The autotuner picks
// the variant per kernel and lattice.
template <int P, int FL, int RED, int MINB = 1, bool ST = false>
__global__ void __launch_bounds__(256, MINB) hop_kernel(const HopArgs a) {
  using R = typename Tr<P>::R;
  const int nrhs = a.nrhs;
  const int rhs = blockIdx.x % nrhs;
  const int sb = blockIdx.x / nrhs;
  const long vh = a.g.vh;
  constexpr int NV = RED == R_NORM ? 1 : RED == R_DOT_A ? 2 : 3;
  PartialSum<R> ps[NV];
  const R beta = pick<R>(a.beta, a.betaf), s1 = pick<R>(a.s1, a.s1f), ca = pick<R>(a.caux, a.cauxf);
  const bool skip = rhs_finished(a.red, rhs);
  if (!skip) {
    const int p = a.out_parity;
    const long lbb = link_block_bytes(P, vh), cbb = clover_block_bytes(P, vh);
    const char* g_out = a.gauge + (long)p * 4 * lbb;
    const char* g_in = a.gauge + (long)(1 - p) * 4 * lbb;
    const char* in = a.in + rhs * a.in_rs;
    const uint32_t stride = (uint32_t)a.nblk * blockDim.x;
    const uint32_t nsite = a.site_map ? a.n_map : (uint32_t)vh;
    for (uint32_t k = sb * blockDim.x + threadIdx.x; k < nsite; k += stride) {
      const uint32_t ih = a.site_map ? __ldg(a.site_map + k) : k;
      int c[4];
      uint32_t xh;
      site_coords(a.g, ih, p, c, xh);
      cx<R> acc[12];
#pragma unroll
      for (int k = 0; k < 12; ++k) acc[k] = czero<R>();
      hop_dir<P, 0, ST>(a, in, g_out, g_in, lbb, ih, c, xh, acc);
      hop_dir<P, 1, ST>(a, in, g_out, g_in, lbb, ih, c, xh, acc);
      hop_dir<P, 2, ST>(a, in, g_out, g_in, lbb, ih, c, xh, acc);
      hop_dir<P, 3, ST>(a, in, g_out, g_in, lbb, ih, c, xh, acc);
#pragma unroll
      for (int k = 0; k < 12; ++k) acc[k] = beta * acc[k];
      if (FL & F_AUX) {
        cx<R> x[12];
        load_spinor<P, true, ST>(a.aux + rhs * a.aux_rs, vh, ih, x);
#pragma unroll
        for (int k = 0; k < 12; ++k) acc[k] = acc[k] + ca * x[k];
      }
      if (FL & F_G5) {
#pragma unroll
        for (int k = 6; k < 12; ++k) acc[k] = cx<R>{-acc[k].r, -acc[k].i};
      }
      cx<R> v[12];
      if (FL & F_E_CLOV) {
        clover_apply<P, ST>(a.clovE + p * cbb, vh, ih, acc, v);
      } else {
#pragma unroll
        for (int k = 0; k < 12; ++k) v[k] = acc[k];
      }
      cx<R> s[12];
      if (FL & F_SELF) {
        load_spinor<P, true, ST>(a.self + rhs * a.self_rs, vh, ih, s);
        if (FL & F_SELF_CLOV) {
          cx<R> ms[12];
          clover_apply<P, ST>(a.clovM + p * cbb, vh, ih, s, ms);
#pragma unroll
          for (int k = 0; k < 12; ++k) v[k] = v[k] + s1 * ms[k];
        } else {
#pragma unroll
          for (int k = 0; k < 12; ++k) v[k] = v[k] + s1 * s[k];
        }
      }
      store_spinor<P>(a.out + rhs * a.out_rs, vh, ih, v);
      if (RED == R_NORM) {
        R n = 0;
#pragma unroll
        for (int k = 0; k < 12; ++k) n += v[k].r * v[k].r + v[k].i * v[k].i;
        ps[0].add(n);
      } else if (RED == R_DOT_A) {
        cx<R> w[12];
        load_spinor<P, true, ST>(a.avec + rhs * a.avec_rs, vh, ih, w);
        cx<R> d = czero<R>();
#pragma unroll
        for (int k = 0; k < 12; ++k) d = d + cmul_conj(w[k], v[k]);
        ps[0].add(d.r);
        ps[1].add(d.i);
      } else if (RED == R_TS) {
        cx<R> d = czero<R>();
        R n = 0;
#pragma unroll
        for (int k = 0; k < 12; ++k) {
          d = d + cmul_conj(v[k], s[k]);
          n += v[k].r * v[k].r + v[k].i * v[k].i;
        }
        ps[0].add(d.r);
        ps[1].add(d.i);
        ps[2].add(n);
      }
    }
  }
  if (RED != R_NONE) {
    double rv[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) rv[k] = ps[k].value();
    reduce_finalize<NV>(a.red, rhs, sb, a.nblk, nrhs, rv);
  }
}

// ---------------------------------------------------------------------------
// NR right-hand sides per thread.  With several right-hand sides the stencil
// is limited by instruction issue rather than by memory, so one thread
// computes one site for NR consecutive right-hand sides and shares among
// them the neighbour indices, the link loads with row-3 reconstruction and
// the clover blocks.  Right-hand sides [r0, r0 + nr) of group g; a
// right-hand side whose solve has finished is skipped (uniform per block).
template <int P, int MU, bool FWD, int NR>
BR_D void hop_one_mr(const char* in, long in_rs, const bool live[NR], const char* lb, long vh, uint32_t nb,
                     uint32_t li, bool wraps, typename Tr<P>::R bc, cx<typename Tr<P>::R> acc[NR][12]) {
  using T = typename Tr<P>::R;
  Link<T> U;
  load_link<P, true>(lb, vh, li, U);
#pragma unroll
  for (int r = 0; r < NR; ++r) {
    if (!live[r]) continue;
    cx<T> h[2][3];
    const char* src = in + r * in_rs;
    if constexpr (Tr<P>::half) {
      cx<float> psi[12];
      const float sc = load_spinor_unscaled<P>(src, vh, nb, psi) * (wraps ? bc : 1.0f);
      project<T, MU, FWD>(psi, h);
#pragma unroll
      for (int k = 0; k < 2; ++k)
#pragma unroll
        for (int c = 0; c < 3; ++c) h[k][c] = sc * h[k][c];
    } else {
      {
        cx<T> psi[12];
        load_spinor<P>(src, vh, nb, psi);
        project<T, MU, FWD>(psi, h);
      }
      if (wraps) {
#pragma unroll
        for (int k = 0; k < 2; ++k)
#pragma unroll
          for (int c = 0; c < 3; ++c) h[k][c] = bc * h[k][c];
      }
    }
    cx<T> u[2][3];
#pragma unroll
    for (int k = 0; k < 2; ++k)
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        if (FWD)
          u[k][q] = crow3(U.m[q][0], U.m[q][1], U.m[q][2], h[k]);
        else
          u[k][q] = crow3_conj(U.m[0][q], U.m[1][q], U.m[2][q], h[k]);
      }
    reconstruct<T, MU, FWD>(u, acc[r]);
  }
}

template <int P, int MU, int NR>
BR_D void hop_dir_mr(const HopArgs& a, const char* in, const bool live[NR], const char* g_out, const char* g_in,
                     long lbb, uint32_t ih, const int c[4], uint32_t xh, cx<typename Tr<P>::R> acc[NR][12]) {
  using T = typename Tr<P>::R;
  uint32_t f, b;
  bool wf, wb;
  neighbours<MU>(a.g, ih, c, xh, f, b, wf, wb);
  const T bc = pick<T>(a.bc[MU], a.bcf[MU]);
  hop_one_mr<P, MU, true, NR>(in, a.in_rs, live, g_out + MU * lbb, a.g.vh, f, ih, wf, bc, acc);
  hop_one_mr<P, MU, false, NR>(in, a.in_rs, live, g_in + MU * lbb, a.g.vh, b, b, wb, bc, acc);
}

template <int P, int FL, int RED, int NR>
__global__ void __launch_bounds__(256) hop_kernel_mr(const HopArgs a) {
  using T = typename Tr<P>::R;
  const int ng = (a.nrhs + NR - 1) / NR;
  const int g = blockIdx.x % ng;
  const int sb = blockIdx.x / ng;
  const int r0 = g * NR;
  const long vh = a.g.vh;
  constexpr int NV = RED == R_NORM ? 1 : RED == R_DOT_A ? 2 : 3;
  bool live[NR];
  bool any = false;
#pragma unroll
  for (int r = 0; r < NR; ++r) {
    live[r] = (r0 + r < a.nrhs) && !rhs_finished(a.red, r0 + r);
    any = any || live[r];
  }
  PartialSum<T> ps[NR][NV];
  const T beta = pick<T>(a.beta, a.betaf), s1 = pick<T>(a.s1, a.s1f), ca = pick<T>(a.caux, a.cauxf);
  if (any) {
    const int p = a.out_parity;
    const long lbb = link_block_bytes(P, vh), cbb = clover_block_bytes(P, vh);
    const char* g_out = a.gauge + (long)p * 4 * lbb;
    const char* g_in = a.gauge + (long)(1 - p) * 4 * lbb;
    const char* in = a.in + r0 * a.in_rs;
    const uint32_t stride = (uint32_t)a.nblk * blockDim.x;
    const uint32_t nsite = a.site_map ? a.n_map : (uint32_t)vh;
    for (uint32_t k = sb * blockDim.x + threadIdx.x; k < nsite; k += stride) {
      const uint32_t ih = a.site_map ? __ldg(a.site_map + k) : k;
      int c[4];
      uint32_t xh;
      site_coords(a.g, ih, p, c, xh);
      cx<T> acc[NR][12];
#pragma unroll
      for (int r = 0; r < NR; ++r)
#pragma unroll
        for (int k = 0; k < 12; ++k) acc[r][k] = czero<T>();
      hop_dir_mr<P, 0, NR>(a, in, live, g_out, g_in, lbb, ih, c, xh, acc);
      hop_dir_mr<P, 1, NR>(a, in, live, g_out, g_in, lbb, ih, c, xh, acc);
      hop_dir_mr<P, 2, NR>(a, in, live, g_out, g_in, lbb, ih, c, xh, acc);
      hop_dir_mr<P, 3, NR>(a, in, live, g_out, g_in, lbb, ih, c, xh, acc);
#pragma unroll
      for (int r = 0; r < NR; ++r) {
#pragma unroll
        for (int k = 0; k < 12; ++k) acc[r][k] = beta * acc[r][k];
        if ((FL & F_AUX) && live[r]) {
          cx<T> x[12];
          load_spinor<P, true, true>(a.aux + (r0 + r) * a.aux_rs, vh, ih, x);
#pragma unroll
          for (int k = 0; k < 12; ++k) acc[r][k] = acc[r][k] + ca * x[k];
        }
      }
      if (FL & F_E_CLOV) {
        // one load of each 6x6 block, applied to every right-hand side
#pragma unroll
        for (int b = 0; b < 2; ++b) {
          T m[36];
          load_clover_block<P, true>(a.clovE + p * cbb, vh, ih, b, m);
#pragma unroll
          for (int r = 0; r < NR; ++r) {
            cx<T> y[6];
            hermitian6_apply<T>(m, acc[r] + 6 * b, y);
#pragma unroll
            for (int k = 0; k < 6; ++k) acc[r][6 * b + k] = y[k];
          }
        }
      }
#pragma unroll
      for (int r = 0; r < NR; ++r) {
        if (!live[r]) continue;
        cx<T> s[12];
        if (FL & F_SELF) {
          load_spinor<P, true, true>(a.self + (r0 + r) * a.self_rs, vh, ih, s);
#pragma unroll
          for (int k = 0; k < 12; ++k) acc[r][k] = acc[r][k] + s1 * s[k];
        }
        store_spinor<P>(a.out + (r0 + r) * a.out_rs, vh, ih, acc[r]);
        if (RED == R_NORM) {
          T n = 0;
#pragma unroll
          for (int k = 0; k < 12; ++k) n += acc[r][k].r * acc[r][k].r + acc[r][k].i * acc[r][k].i;
          ps[r][0].add(n);
        } else if (RED == R_DOT_A) {
          cx<T> w[12];
          load_spinor<P, true, true>(a.avec + (r0 + r) * a.avec_rs, vh, ih, w);
          cx<T> d = czero<T>();
#pragma unroll
          for (int k = 0; k < 12; ++k) d = d + cmul_conj(w[k], acc[r][k]);
          ps[r][0].add(d.r);
          ps[r][1].add(d.i);
        } else if (RED == R_TS) {
          cx<T> d = czero<T>();
          T n = 0;
#pragma unroll
          for (int k = 0; k < 12; ++k) {
            d = d + cmul_conj(acc[r][k], s[k]);
            n += acc[r][k].r * acc[r][k].r + acc[r][k].i * acc[r][k].i;
          }
          ps[r][0].add(d.r);
          ps[r][1].add(d.i);
          ps[r][2].add(n);
        }
      }
    }
  }
  if (RED != R_NONE) {
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      if (r0 + r >= a.nrhs) break;  // uniform per block
      double rv[NV];
#pragma unroll
      for (int k = 0; k < NV; ++k) rv[k] = ps[r][k].value();
      block_partial<NV>(a.red, r0 + r, sb, a.nblk, rv);
    }
    grid_finish<NV>(a.red, a.nblk, a.nrhs);
  }
}

// Launch with the given block size on a stream; returns false for a
// (flags, reduction) pair that is not instantiated.  With occ != null,
// nothing is launched: *occ receives the resident blocks per SM instead.
// variant v in [0, 6): register budget {none, 80, 64}[v % 3] and, for v >= 3,
// read-once operands loaded around L1; v in {6, 7, 8}: 2, 3 or 4 right-hand
// sides per thread (hop_kernel_mr; grid = nblk x ceil(nrhs / NR)); v in
// {9, 10}: the shared-link tile kernel (hop_kernel_tile, 32-site tiles for
// up to 12 right-hand sides per block, one / two tiles staged per barrier;
// grid = nblk x ceil(nrhs / 12), the block size is its own).
// Only the kernels of the Schur passes, D_eo and the FP64 residual have
// variants other than 0, and only FP32/FP16/BF16 have the multi-RHS ones.
template <int P>
bool launch_hop(int flags, int red, const HopArgs& a, int block, cudaStream_t st, int* occ = nullptr, int variant = 0);
template <>
bool launch_hop<P_F64>(int flags, int red, const HopArgs& a, int block, cudaStream_t st, int* occ, int variant);
template <>
bool launch_hop<P_F32>(int flags, int red, const HopArgs& a, int block, cudaStream_t st, int* occ, int variant);
template <>
bool launch_hop<P_F16>(int flags, int red, const HopArgs& a, int block, cudaStream_t st, int* occ, int variant);
template <>
bool launch_hop<P_BF16>(int flags, int red, const HopArgs& a, int block, cudaStream_t st, int* occ, int variant);
bool hop_has_variants(int flags, int red);
// Right-hand sides covered by one block group of a variant: 1 for v < 6, NR
// for the NR-per-thread kernels (v = 6, 7, 8) and up to 12 for the
// shared-link tile kernels (v = 9, 10; with pipelined neighbour loads, 16-bit
// storage only, v = 11, 12; dslash_tile.cuh).
inline int hop_variant_rpt(int variant) { return variant >= 9 ? 12 : variant >= 6 ? variant - 4 : 1; }
constexpr int HOP_NVARIANT = 13;
inline bool hop_variant_for_prec(int variant, int prec) { return variant < 11 || prec == P_F16 || prec == P_BF16; }
inline bool hop_variant_is_tile(int variant) { return variant >= 9; }

}  // namespace bridge
