// Staggered operator kernels.
//
// Operator (Sec. 2 of the paper implements the staggered action and its
// even-odd blocks, Eq. 1; the formula is the textbook Kogut-Susskind one):
//   D chi(x) = m chi(x) + (1/2) sum_mu eta_mu(x) [ U_mu(x) chi(x + mu)
//                                               - U_mu(x - mu)^dagger chi(x - mu) ]
// with eta_0 = 1, eta_1 = (-1)^x, eta_2 = (-1)^(x+y), eta_3 = (-1)^(x+y+z) and
// the boundary phase bc[mu] on every hop that wraps.  The phases are applied
// in the kernel; the links are the same stored links as for Wilson (FP64 18
// reals, FP32 12 reals with row 2 rebuilt in registers).
//
// Field layout: a half-lattice colour vector is three 8-byte (FP32) or
// 16-byte (FP64) planes, one complex colour component each, addressed
// base + (k * Vh + ih) * size, so a warp reads contiguous bytes per plane.
//
// One thread computes one output site of one right-hand side:
//   out = scale * sum_mu eta_mu [U chi(x+mu) - U^dag chi(x-mu)] + s1 self + caux aux
// with an optional fused reduction of |out|^2 or Re <self, out>.
#pragma once

#include "common.cuh"
#include "reduce.cuh"

namespace bridge {

BR_HD long stag_site_bytes(int prec) { return prec == P_F64 ? 48 : 24; }
BR_HD long stag_block_bytes(int prec, long vh) { return pad256(stag_site_bytes(prec) * vh); }

template <int P>
BR_D void load_cvec(const char* base, long vh, uint32_t i, cx<typename Tr<P>::R> v[3]) {
  if constexpr (P == P_F64) {
    const double2* p = reinterpret_cast<const double2*>(base);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const double2 w = __ldg(p + k * vh + i);
      v[k] = {w.x, w.y};
    }
  } else {
    const float2* p = reinterpret_cast<const float2*>(base);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const float2 w = __ldg(p + k * vh + i);
      v[k] = {w.x, w.y};
    }
  }
}

// Plain (coherent) load, for vectors this kernel also writes.
template <int P>
BR_D void load_cvec_rw(const char* base, long vh, uint32_t i, cx<typename Tr<P>::R> v[3]) {
  if constexpr (P == P_F64) {
    const double2* p = reinterpret_cast<const double2*>(base);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const double2 w = p[k * vh + i];
      v[k] = {w.x, w.y};
    }
  } else {
    const float2* p = reinterpret_cast<const float2*>(base);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const float2 w = p[k * vh + i];
      v[k] = {w.x, w.y};
    }
  }
}

template <int P>
BR_D void store_cvec(char* base, long vh, uint32_t i, const cx<typename Tr<P>::R> v[3]) {
  if constexpr (P == P_F64) {
    double2* p = reinterpret_cast<double2*>(base);
#pragma unroll
    for (int k = 0; k < 3; ++k) p[k * vh + i] = make_double2(v[k].r, v[k].i);
  } else {
    float2* p = reinterpret_cast<float2*>(base);
#pragma unroll
    for (int k = 0; k < 3; ++k) p[k * vh + i] = make_float2(v[k].r, v[k].i);
  }
}

enum StagRed { SR_NONE = 0, SR_NORM = 1, SR_DOT_SELF = 2 };

struct StagArgs {
  Geom g;
  int out_parity, nrhs, nblk;
  double scale, s1, caux;
  float scalef, s1f, cauxf;
  double bc[4];
  float bcf[4];
  char* out;
  long out_rs;
  const char* in;
  long in_rs;
  const char* self;  // may be null
  long self_rs;
  const char* aux;   // may be null
  long aux_rs;
  const char* gauge;  // [parity][mu] link blocks
  RedArgs red;
};

template <int P, int MU, bool FWD>
BR_D void stag_hop_one(const char* in, const char* lb, long vh, uint32_t nb, uint32_t li, bool wraps,
                       typename Tr<P>::R bc, typename Tr<P>::R eta, cx<typename Tr<P>::R> acc[3]) {
  using R = typename Tr<P>::R;
  cx<R> v[3];
  load_cvec<P>(in, vh, nb, v);
  Link<R> U;
  load_link<P, true>(lb, vh, li, U);
  const R f = (wraps ? bc : R(1)) * (FWD ? eta : -eta);
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    cx<R> w;
    if (FWD)
      w = crow3(U.m[r][0], U.m[r][1], U.m[r][2], v);
    else
      w = crow3_conj(U.m[0][r], U.m[1][r], U.m[2][r], v);
    acc[r] = caxpy(f, w, acc[r]);
  }
}

template <int P, int MU>
BR_D void stag_dir(const StagArgs& a, const char* in, const char* g_out, const char* g_in, long lbb, uint32_t ih,
                   const int c[4], uint32_t xh, typename Tr<P>::R eta, cx<typename Tr<P>::R> acc[3]) {
  using R = typename Tr<P>::R;
  uint32_t f, b;
  bool wf, wb;
  neighbours<MU>(a.g, ih, c, xh, f, b, wf, wb);
  const R bc = pick<R>(a.bc[MU], a.bcf[MU]);
  stag_hop_one<P, MU, true>(in, g_out + MU * lbb, a.g.vh, f, ih, wf, bc, eta, acc);
  stag_hop_one<P, MU, false>(in, g_in + MU * lbb, a.g.vh, b, b, wb, bc, eta, acc);
}

template <int P, int RED>
__global__ void __launch_bounds__(256) stag_hop_kernel(const StagArgs a) {
  using R = typename Tr<P>::R;
  const int nrhs = a.nrhs;
  const int rhs = blockIdx.x % nrhs;
  const int sb = blockIdx.x / nrhs;
  const long vh = a.g.vh;
  PartialSum<R> ps;
  const bool skip = a.red.check_done && a.red.cg != nullptr && a.red.cg[rhs].done != RUNNING;
  if (!skip) {
    const int p = a.out_parity;
    const long lbb = link_block_bytes(P, vh);
    const char* g_out = a.gauge + (long)p * 4 * lbb;
    const char* g_in = a.gauge + (long)(1 - p) * 4 * lbb;
    const char* in = a.in + rhs * a.in_rs;
    const R sc = pick<R>(a.scale, a.scalef), s1 = pick<R>(a.s1, a.s1f), ca = pick<R>(a.caux, a.cauxf);
    const uint32_t stride = (uint32_t)a.nblk * blockDim.x;
    for (uint32_t ih = sb * blockDim.x + threadIdx.x; ih < (uint32_t)vh; ih += stride) {
      int c[4];
      uint32_t xh;
      site_coords(a.g, ih, p, c, xh);
      cx<R> acc[3] = {czero<R>(), czero<R>(), czero<R>()};
      stag_dir<P, 0>(a, in, g_out, g_in, lbb, ih, c, xh, R(1), acc);
      stag_dir<P, 1>(a, in, g_out, g_in, lbb, ih, c, xh, (c[0] & 1) ? R(-1) : R(1), acc);
      stag_dir<P, 2>(a, in, g_out, g_in, lbb, ih, c, xh, ((c[0] + c[1]) & 1) ? R(-1) : R(1), acc);
      stag_dir<P, 3>(a, in, g_out, g_in, lbb, ih, c, xh, ((c[0] + c[1] + c[2]) & 1) ? R(-1) : R(1), acc);
      cx<R> v[3], s[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) v[k] = sc * acc[k];
      if (a.self != nullptr) {
        load_cvec<P>(a.self + rhs * a.self_rs, vh, ih, s);
#pragma unroll
        for (int k = 0; k < 3; ++k) v[k] = v[k] + s1 * s[k];
      }
      if (a.aux != nullptr) {
        cx<R> w[3];
        load_cvec<P>(a.aux + rhs * a.aux_rs, vh, ih, w);
#pragma unroll
        for (int k = 0; k < 3; ++k) v[k] = v[k] + ca * w[k];
      }
      store_cvec<P>(a.out + rhs * a.out_rs, vh, ih, v);
      if (RED == SR_NORM) {
        R n = 0;
#pragma unroll
        for (int k = 0; k < 3; ++k) n += v[k].r * v[k].r + v[k].i * v[k].i;
        ps.add(n);
      } else if (RED == SR_DOT_SELF) {
        R d = 0;
#pragma unroll
        for (int k = 0; k < 3; ++k) d += s[k].r * v[k].r + s[k].i * v[k].i;
        ps.add(d);
      }
    }
  }
  if (RED != SR_NONE) {
    double rv[1] = {ps.value()};
    reduce_finalize<1>(a.red, rhs, sb, a.nblk, nrhs, rv);
  }
}

// ------------------------------------------------------------ vector kernels
enum StagVecOp {
  SV_CGUPD = 0,   // x += alpha p, r -= alpha q, |r|^2 -> FIN_CG_BETA
  SV_CGP = 1,     // p = r + beta p
  SV_NORM = 2,    // |a|^2 -> red.fin
  SV_CONVERT = 3, // b (precision PB) = mask ? a (precision P) : 0
  SV_ACCUM = 4,   // b (FP64) += mask ? a : 0
  SV_FROM_CANON = 5,
  SV_TO_CANON = 6
};

struct StagVecArgs {
  Geom g;
  uint32_t vh;
  int nrhs, nblk, parity;
  long V;             // full volume (canonical strides)
  int canon_full;     // 1: canonical full-lattice vectors; 0: half-lattice (site ih of this parity)
  char *a, *b, *c, *d;  // operands (see StagVecOp)
  long a_rs, b_rs, c_rs, d_rs;
  double* canon;      // canonical FP64 full-lattice vectors (V * 6 doubles per rhs)
  const int* mask;    // per rhs (may be null)
  RedArgs red;
};

template <int P, int PB, int OP>
__global__ void __launch_bounds__(256) stag_vec_kernel(const StagVecArgs a) {
  using R = typename Tr<P>::R;
  using RB = typename Tr<PB>::R;
  const int rhs = blockIdx.x % a.nrhs;
  const int sb = blockIdx.x / a.nrhs;
  PartialSum<R> ps;
  const bool skip = (OP == SV_CGUPD || OP == SV_CGP) && a.red.cg != nullptr && a.red.cg[rhs].done != RUNNING;
  const bool on = a.mask == nullptr || a.mask[rhs] != 0;
  if (!skip) {
    const uint32_t stride = (uint32_t)a.nblk * blockDim.x;
    for (uint32_t ih = sb * blockDim.x + threadIdx.x; ih < a.vh; ih += stride) {
      if (OP == SV_CGUPD) {
        const R alpha = (R)a.red.cg[rhs].alpha;
        cx<R> x[3], r[3], p[3], q[3];
        load_cvec_rw<P>(a.a + rhs * a.a_rs, a.vh, ih, x);
        load_cvec_rw<P>(a.b + rhs * a.b_rs, a.vh, ih, r);
        load_cvec<P>(a.c + rhs * a.c_rs, a.vh, ih, p);
        load_cvec<P>(a.d + rhs * a.d_rs, a.vh, ih, q);
        R n = 0;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          x[k] = x[k] + alpha * p[k];
          r[k] = r[k] - alpha * q[k];
          n += r[k].r * r[k].r + r[k].i * r[k].i;
        }
        store_cvec<P>(a.a + rhs * a.a_rs, a.vh, ih, x);
        store_cvec<P>(a.b + rhs * a.b_rs, a.vh, ih, r);
        ps.add(n);
      } else if (OP == SV_CGP) {
        const R beta = (R)a.red.cg[rhs].beta;
        cx<R> p[3], r[3];
        load_cvec_rw<P>(a.a + rhs * a.a_rs, a.vh, ih, p);
        load_cvec<P>(a.b + rhs * a.b_rs, a.vh, ih, r);
#pragma unroll
        for (int k = 0; k < 3; ++k) p[k] = r[k] + beta * p[k];
        store_cvec<P>(a.a + rhs * a.a_rs, a.vh, ih, p);
      } else if (OP == SV_NORM) {
        cx<R> v[3];
        load_cvec<P>(a.a + rhs * a.a_rs, a.vh, ih, v);
        R n = 0;
#pragma unroll
        for (int k = 0; k < 3; ++k) n += v[k].r * v[k].r + v[k].i * v[k].i;
        ps.add(n);
      } else if (OP == SV_CONVERT) {
        cx<R> v[3];
        cx<RB> w[3];
        load_cvec<P>(a.a + rhs * a.a_rs, a.vh, ih, v);
#pragma unroll
        for (int k = 0; k < 3; ++k) w[k] = on ? cx<RB>{(RB)v[k].r, (RB)v[k].i} : czero<RB>();
        store_cvec<PB>(a.b + rhs * a.b_rs, a.vh, ih, w);
      } else if (OP == SV_ACCUM) {
        if (!on) continue;
        cx<R> v[3];
        cx<double> w[3];
        load_cvec<P>(a.a + rhs * a.a_rs, a.vh, ih, v);
        load_cvec_rw<P_F64>(a.b + rhs * a.b_rs, a.vh, ih, w);
#pragma unroll
        for (int k = 0; k < 3; ++k) w[k] = w[k] + cx<double>{(double)v[k].r, (double)v[k].i};
        store_cvec<P_F64>(a.b + rhs * a.b_rs, a.vh, ih, w);
      } else {
        int c[4];
        uint32_t xh;
        site_coords(a.g, ih, a.parity, c, xh);
        const long site = c[0] + (long)a.g.L[0] * (c[1] + (long)a.g.L[1] * (c[2] + (long)a.g.L[2] * c[3]));
        double* cp = a.canon_full ? a.canon + ((long)rhs * a.V + site) * 6 : a.canon + ((long)rhs * a.vh + ih) * 6;
        if (OP == SV_FROM_CANON) {
          cx<R> v[3];
#pragma unroll
          for (int k = 0; k < 3; ++k) v[k] = {(R)cp[2 * k], (R)cp[2 * k + 1]};
          store_cvec<P>(a.a + rhs * a.a_rs, a.vh, ih, v);
        } else {
          cx<R> v[3];
          load_cvec<P>(a.a + rhs * a.a_rs, a.vh, ih, v);
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            cp[2 * k] = (double)v[k].r;
            cp[2 * k + 1] = (double)v[k].i;
          }
        }
      }
    }
  }
  if (OP == SV_CGUPD || OP == SV_NORM) {
    double rv[1] = {ps.value()};
    reduce_finalize<1>(a.red, rhs, sb, a.nblk, a.nrhs, rv);
  }
}

}  // namespace bridge
