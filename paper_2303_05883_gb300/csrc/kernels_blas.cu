// BiCGStab vector kernels (fused updates + reductions), layout conversions
// between the canonical FP64 host layout and the GPU site layout, and the
// site-local clover product.  All are bandwidth-bound one-pass kernels: one
// thread per site (per right-hand side), 16-byte plane accesses.
#include "kernels.h"

namespace bridge {

#define BR_SITE_LOOP(vh_, nblk_) \
  for (uint32_t ih = (uint32_t)(blockIdx.x / a.nrhs) * blockDim.x + threadIdx.x; ih < (vh_); ih += (uint32_t)(nblk_) * blockDim.x)

template <class R>
BR_D cx<R> scal(cx<R> z, cx<R> v) {  // z * v
  return {z.r * v.r - z.i * v.i, z.r * v.i + z.i * v.r};
}

// ------------------------------------------------------------- BiCGStab
template <int P, int PX>
__global__ void __launch_bounds__(256) k_blas_init(const BlasArgs a) {
  using R = typename Tr<P>::R;
  const int rhs = blockIdx.x % a.nrhs, sb = blockIdx.x / a.nrhs;
  PartialSum<R> ps;
  BR_SITE_LOOP(a.vh, a.nblk) {
    cx<R> b[12], z[12];
    load_spinor<P>(a.b + rhs * a.b_rs, a.vh, ih, b);
    R n = 0;
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      n += b[k].r * b[k].r + b[k].i * b[k].i;
      z[k] = czero<R>();
    }
    store_spinor<P>(a.r + rhs * a.r_rs, a.vh, ih, b);
    store_spinor<P>(a.rhat + rhs * a.rhat_rs, a.vh, ih, b);
    store_spinor<P>(a.p + rhs * a.p_rs, a.vh, ih, b);
    store_spinor<PX>(a.x + rhs * a.x_rs, a.vh, ih, z);
    ps.add(n);
  }
  double rv[1] = {ps.value()};
  reduce_finalize<1>(a.red, rhs, sb, a.nblk, a.nrhs, rv);
}

template <int P>
__global__ void __launch_bounds__(256) k_blas_s(const BlasArgs a) {
  using R = typename Tr<P>::R;
  const int rhs = blockIdx.x % a.nrhs;
  const BiCGScalars* q = a.red.sc + rhs;
  if (q->done != RUNNING) return;
  const cx<R> al = {(R)q->alpha_r, (R)q->alpha_i};
  BR_SITE_LOOP(a.vh, a.nblk) {
    cx<R> r[12], v[12];
    load_spinor<P, false>(a.r + rhs * a.r_rs, a.vh, ih, r);
    load_spinor<P, false>(a.v + rhs * a.v_rs, a.vh, ih, v);
#pragma unroll
    for (int k = 0; k < 12; ++k) r[k] = r[k] - scal<R>(al, v[k]);
    store_spinor<P>(a.s + rhs * a.s_rs, a.vh, ih, r);
  }
}

template <int P, int PX>
__global__ void __launch_bounds__(256) k_blas_xr(const BlasArgs a) {
  using R = typename Tr<P>::R;
  const int rhs = blockIdx.x % a.nrhs, sb = blockIdx.x / a.nrhs;
  const BiCGScalars* q = a.red.sc + rhs;
  PartialSum<R> ps[3];
  if (q->done == RUNNING) {
    const cx<R> al = {(R)q->alpha_r, (R)q->alpha_i}, om = {(R)q->omega_r, (R)q->omega_i};
    BR_SITE_LOOP(a.vh, a.nblk) {
      cx<R> x[12], p[12], s[12], t[12];
      load_spinor<PX, false>(a.x + rhs * a.x_rs, a.vh, ih, x);
      load_spinor<P, false>(a.p + rhs * a.p_rs, a.vh, ih, p);
      load_spinor<P, false>(a.s + rhs * a.s_rs, a.vh, ih, s);
#pragma unroll
      for (int k = 0; k < 12; ++k) x[k] = x[k] + scal<R>(al, p[k]) + scal<R>(om, s[k]);
      store_spinor<PX>(a.x + rhs * a.x_rs, a.vh, ih, x);
      load_spinor<P, false>(a.t + rhs * a.t_rs, a.vh, ih, t);
#pragma unroll
      for (int k = 0; k < 12; ++k) s[k] = s[k] - scal<R>(om, t[k]);  // new r
      store_spinor<P>(a.r + rhs * a.r_rs, a.vh, ih, s);
      load_spinor<P, false>(a.rhat + rhs * a.rhat_rs, a.vh, ih, p);
      cx<R> d = czero<R>();
      R n = 0;
#pragma unroll
      for (int k = 0; k < 12; ++k) {
        d = d + cmul_conj(p[k], s[k]);
        n += s[k].r * s[k].r + s[k].i * s[k].i;
      }
      ps[0].add(d.r);
      ps[1].add(d.i);
      ps[2].add(n);
    }
  }
  double rv[3] = {ps[0].value(), ps[1].value(), ps[2].value()};
  reduce_finalize<3>(a.red, rhs, sb, a.nblk, a.nrhs, rv);
}

template <int P>
__global__ void __launch_bounds__(256) k_blas_p(const BlasArgs a) {
  using R = typename Tr<P>::R;
  const int rhs = blockIdx.x % a.nrhs;
  const BiCGScalars* q = a.red.sc + rhs;
  if (q->done != RUNNING) return;
  const cx<R> be = {(R)q->beta_r, (R)q->beta_i}, om = {(R)q->omega_r, (R)q->omega_i};
  BR_SITE_LOOP(a.vh, a.nblk) {
    cx<R> r[12], p[12], v[12];
    load_spinor<P, false>(a.r + rhs * a.r_rs, a.vh, ih, r);
    load_spinor<P, false>(a.p + rhs * a.p_rs, a.vh, ih, p);
    load_spinor<P, false>(a.v + rhs * a.v_rs, a.vh, ih, v);
#pragma unroll
    for (int k = 0; k < 12; ++k) p[k] = r[k] + scal<R>(be, p[k] - scal<R>(om, v[k]));
    store_spinor<P>(a.p + rhs * a.p_rs, a.vh, ih, p);
  }
}

// ----------------------------------------------------------- CG on D^dag D^
// CG (Hestenes-Stiefel) on the normal equations of the Schur system, the
// inner method where BiCGStab stagnates (a spectrum around the origin past
// the critical kappa); real scalars from CGScalars (FIN_CG_* finalizers):
// B_CG_INIT x = 0, p = r, |r|^2 -> FIN_CG_INIT
// B_CG_XR   x += alpha p, r -= alpha t, |r|^2 -> FIN_CG_BETA
// B_CG_P    p = r + beta p
template <int P, int PX>
__global__ void __launch_bounds__(256) k_cg_init(const BlasArgs a) {
  using R = typename Tr<P>::R;
  const int rhs = blockIdx.x % a.nrhs, sb = blockIdx.x / a.nrhs;
  PartialSum<R> ps;
  BR_SITE_LOOP(a.vh, a.nblk) {
    cx<R> r[12], z[12];
    load_spinor<P>(a.r + rhs * a.r_rs, a.vh, ih, r);
    R n = 0;
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      n += r[k].r * r[k].r + r[k].i * r[k].i;
      z[k] = czero<R>();
    }
    store_spinor<P>(a.p + rhs * a.p_rs, a.vh, ih, r);
    store_spinor<PX>(a.x + rhs * a.x_rs, a.vh, ih, z);
    ps.add(n);
  }
  double rv[1] = {ps.value()};
  reduce_finalize<1>(a.red, rhs, sb, a.nblk, a.nrhs, rv);
}

template <int P, int PX>
__global__ void __launch_bounds__(256) k_cg_xr(const BlasArgs a) {
  using R = typename Tr<P>::R;
  const int rhs = blockIdx.x % a.nrhs, sb = blockIdx.x / a.nrhs;
  const CGScalars* q = a.red.cg + rhs;
  PartialSum<R> ps;
  if (q->done == RUNNING) {
    const R al = (R)q->alpha;
    BR_SITE_LOOP(a.vh, a.nblk) {
      cx<R> x[12], p[12], r[12], t[12];
      load_spinor<PX, false>(a.x + rhs * a.x_rs, a.vh, ih, x);
      load_spinor<P, false>(a.p + rhs * a.p_rs, a.vh, ih, p);
#pragma unroll
      for (int k = 0; k < 12; ++k) x[k] = caxpy(al, p[k], x[k]);
      store_spinor<PX>(a.x + rhs * a.x_rs, a.vh, ih, x);
      load_spinor<P, false>(a.r + rhs * a.r_rs, a.vh, ih, r);
      load_spinor<P, false>(a.t + rhs * a.t_rs, a.vh, ih, t);
      R n = 0;
#pragma unroll
      for (int k = 0; k < 12; ++k) {
        r[k] = caxpy(-al, t[k], r[k]);
        n += r[k].r * r[k].r + r[k].i * r[k].i;
      }
      store_spinor<P>(a.r + rhs * a.r_rs, a.vh, ih, r);
      ps.add(n);
    }
  }
  double rv[1] = {ps.value()};
  reduce_finalize<1>(a.red, rhs, sb, a.nblk, a.nrhs, rv);
}

template <int P>
__global__ void __launch_bounds__(256) k_cg_p(const BlasArgs a) {
  using R = typename Tr<P>::R;
  const int rhs = blockIdx.x % a.nrhs;
  const CGScalars* q = a.red.cg + rhs;
  if (q->done != RUNNING) return;
  const R be = (R)q->beta;
  BR_SITE_LOOP(a.vh, a.nblk) {
    cx<R> r[12], p[12];
    load_spinor<P, false>(a.r + rhs * a.r_rs, a.vh, ih, r);
    load_spinor<P, false>(a.p + rhs * a.p_rs, a.vh, ih, p);
#pragma unroll
    for (int k = 0; k < 12; ++k) p[k] = caxpy(be, p[k], r[k]);
    store_spinor<P>(a.p + rhs * a.p_rs, a.vh, ih, p);
  }
}

template <int P, int PX>
static bool blas_dispatch(int op, const BlasArgs& a, int block, cudaStream_t st, int* occ) {
  const dim3 grid((unsigned)(a.nblk * a.nrhs));
  if (occ) {
    cudaError_t e = cudaErrorInvalidValue;
    switch (op) {
      case B_INIT: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, k_blas_init<P, PX>, block, 0); break;
      case B_S: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, k_blas_s<P>, block, 0); break;
      case B_XR: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, k_blas_xr<P, PX>, block, 0); break;
      case B_P: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, k_blas_p<P>, block, 0); break;
      case B_CG_INIT: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, k_cg_init<P, PX>, block, 0); break;
      case B_CG_XR: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, k_cg_xr<P, PX>, block, 0); break;
      case B_CG_P: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, k_cg_p<P>, block, 0); break;
    }
    return e == cudaSuccess;
  }
  switch (op) {
    case B_INIT: k_blas_init<P, PX><<<grid, block, 0, st>>>(a); return true;
    case B_S: k_blas_s<P><<<grid, block, 0, st>>>(a); return true;
    case B_XR: k_blas_xr<P, PX><<<grid, block, 0, st>>>(a); return true;
    case B_P: k_blas_p<P><<<grid, block, 0, st>>>(a); return true;
    case B_CG_INIT: k_cg_init<P, PX><<<grid, block, 0, st>>>(a); return true;
    case B_CG_XR: k_cg_xr<P, PX><<<grid, block, 0, st>>>(a); return true;
    case B_CG_P: k_cg_p<P><<<grid, block, 0, st>>>(a); return true;
  }
  return false;
}

bool launch_blas(int op, int prec, int px, const BlasArgs& a, int block, cudaStream_t st, int* occ) {
  if (prec == P_F64 && px == P_F64) return blas_dispatch<P_F64, P_F64>(op, a, block, st, occ);
  if (prec == P_F32 && px == P_F32) return blas_dispatch<P_F32, P_F32>(op, a, block, st, occ);
  if (prec == P_F16 && px == P_F32) return blas_dispatch<P_F16, P_F32>(op, a, block, st, occ);
  if (prec == P_BF16 && px == P_F32) return blas_dispatch<P_BF16, P_F32>(op, a, block, st, occ);
  return false;
}

// --------------------------------------------------------------- layout
BR_D long canon_site(const CopyArgs& a, uint32_t ih) {
  if (!a.canon_full) return ih;
  int c[4];
  uint32_t xh;
  site_coords(a.g, ih, a.parity, c, xh);
  return 2 * (long)ih + (c[0] & 1);  // lexicographic index of the site
}

template <int P>
__global__ void __launch_bounds__(256) k_canon_to_field(const CopyArgs a) {
  using R = typename Tr<P>::R;
  const int rhs = blockIdx.x % a.nrhs;
  const bool on = a.mask == nullptr || a.mask[rhs] != 0;
  const long n_sites = a.canon_full ? a.V : (long)a.vh;
  BR_SITE_LOOP(a.vh, a.nblk) {
    const long crs = a.canon_rs ? a.canon_rs : n_sites * 12;
    const double2* src = reinterpret_cast<const double2*>(a.canon) + (long)rhs * crs + canon_site(a, ih) * 12;
    cx<R> s[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      double2 v = on ? __ldg(src + k) : make_double2(0.0, 0.0);
      s[k] = {(R)v.x, (R)v.y};
    }
    store_spinor<P>(a.dst + rhs * a.dst_rs, a.vh, ih, s);
  }
}

template <int P>
__global__ void __launch_bounds__(256) k_field_to_canon(const CopyArgs a) {
  using R = typename Tr<P>::R;
  const int rhs = blockIdx.x % a.nrhs;
  const long n_sites = a.canon_full ? a.V : (long)a.vh;
  BR_SITE_LOOP(a.vh, a.nblk) {
    cx<R> s[12];
    load_spinor<P>(a.src + rhs * a.src_rs, a.vh, ih, s);
    const long crs = a.canon_rs ? a.canon_rs : n_sites * 12;
    double2* dst = reinterpret_cast<double2*>(a.canon_out) + (long)rhs * crs + canon_site(a, ih) * 12;
#pragma unroll
    for (int k = 0; k < 12; ++k) dst[k] = make_double2((double)s[k].r, (double)s[k].i);
  }
}

template <int PS, int PD>
__global__ void __launch_bounds__(256) k_convert(const CopyArgs a) {
  using RS = typename Tr<PS>::R;
  using RD = typename Tr<PD>::R;
  const int rhs = blockIdx.x % a.nrhs;
  const bool on = a.mask == nullptr || a.mask[rhs] != 0;
  BR_SITE_LOOP(a.vh, a.nblk) {
    cx<RS> s[12];
    cx<RD> d[12];
    if (on) load_spinor<PS>(a.src + rhs * a.src_rs, a.vh, ih, s);
#pragma unroll
    for (int k = 0; k < 12; ++k) d[k] = on ? cx<RD>{(RD)s[k].r, (RD)s[k].i} : czero<RD>();
    store_spinor<PD>(a.dst + rhs * a.dst_rs, a.vh, ih, d);
  }
}

template <int PS>
__global__ void __launch_bounds__(256) k_accumulate64(const CopyArgs a) {
  using RS = typename Tr<PS>::R;
  const int rhs = blockIdx.x % a.nrhs;
  if (a.mask != nullptr && a.mask[rhs] == 0) return;
  BR_SITE_LOOP(a.vh, a.nblk) {
    cx<RS> e[12];
    cx<double> x[12];
    load_spinor<PS>(a.src + rhs * a.src_rs, a.vh, ih, e);
    load_spinor<P_F64, false>(a.dst + rhs * a.dst_rs, a.vh, ih, x);
#pragma unroll
    for (int k = 0; k < 12; ++k) x[k] = x[k] + cx<double>{(double)e[k].r, (double)e[k].i};
    store_spinor<P_F64>(a.dst + rhs * a.dst_rs, a.vh, ih, x);
  }
}

template <int P>
__global__ void __launch_bounds__(256) k_norm2(const CopyArgs a) {
  using R = typename Tr<P>::R;
  const int rhs = blockIdx.x % a.nrhs, sb = blockIdx.x / a.nrhs;
  PartialSum<R> ps;
  BR_SITE_LOOP(a.vh, a.nblk) {
    cx<R> s[12];
    load_spinor<P>(a.src + rhs * a.src_rs, a.vh, ih, s);
    R n = 0;
#pragma unroll
    for (int k = 0; k < 12; ++k) n += s[k].r * s[k].r + s[k].i * s[k].i;
    ps.add(n);
  }
  double rv[1] = {ps.value()};
  reduce_finalize<1>(a.red, rhs, sb, a.nblk, a.nrhs, rv);
}

template <int P>
__global__ void __launch_bounds__(256) k_clover_site(const CopyArgs a, const char* clov) {
  using R = typename Tr<P>::R;
  const int rhs = blockIdx.x % a.nrhs;
  BR_SITE_LOOP(a.vh, a.nblk) {
    cx<R> s[12], d[12];
    load_spinor<P>(a.src + rhs * a.src_rs, a.vh, ih, s);
    clover_apply<P>(clov, a.vh, ih, s, d);
    store_spinor<P>(a.dst + rhs * a.dst_rs, a.vh, ih, d);
  }
}

// dst = gamma5 A src (A the site term at each site, or 1 with clov = null);
// gamma5 = diag(1, 1, -1, -1) in the chiral basis commutes with A.
template <int P>
__global__ void __launch_bounds__(256) k_g5_site(const CopyArgs a, const char* clov) {
  using R = typename Tr<P>::R;
  const int rhs = blockIdx.x % a.nrhs;
  if (a.red.cg != nullptr && a.red.check_done && a.red.cg[rhs].done != RUNNING) return;
  BR_SITE_LOOP(a.vh, a.nblk) {
    cx<R> s[12], d[12];
    load_spinor<P>(a.src + rhs * a.src_rs, a.vh, ih, s);
    if (clov) {
      clover_apply<P>(clov, a.vh, ih, s, d);
    } else {
#pragma unroll
      for (int k = 0; k < 12; ++k) d[k] = s[k];
    }
#pragma unroll
    for (int k = 6; k < 12; ++k) d[k] = cx<R>{-d[k].r, -d[k].i};
    store_spinor<P>(a.dst + rhs * a.dst_rs, a.vh, ih, d);
  }
}

#define BR_PREC_SWITCH(prec, KERNEL, ...)                                                    \
  switch (prec) {                                                                             \
    case P_F64: KERNEL<P_F64><<<grid, block, 0, st>>>(__VA_ARGS__); return true;             \
    case P_F32: KERNEL<P_F32><<<grid, block, 0, st>>>(__VA_ARGS__); return true;             \
    case P_F16: KERNEL<P_F16><<<grid, block, 0, st>>>(__VA_ARGS__); return true;             \
    case P_BF16: KERNEL<P_BF16><<<grid, block, 0, st>>>(__VA_ARGS__); return true;           \
  }                                                                                           \
  return false;

bool launch_canon_to_field(int prec, const CopyArgs& a, int block, cudaStream_t st) {
  const dim3 grid((unsigned)(a.nblk * a.nrhs));
  BR_PREC_SWITCH(prec, k_canon_to_field, a)
}
bool launch_field_to_canon(int prec, const CopyArgs& a, int block, cudaStream_t st) {
  const dim3 grid((unsigned)(a.nblk * a.nrhs));
  BR_PREC_SWITCH(prec, k_field_to_canon, a)
}
bool launch_accumulate64(int prec, const CopyArgs& a, int block, cudaStream_t st) {
  const dim3 grid((unsigned)(a.nblk * a.nrhs));
  BR_PREC_SWITCH(prec, k_accumulate64, a)
}
bool launch_norm2(int prec, const CopyArgs& a, int block, cudaStream_t st) {
  const dim3 grid((unsigned)(a.nblk * a.nrhs));
  BR_PREC_SWITCH(prec, k_norm2, a)
}
bool launch_clover_site(int prec, const CopyArgs& a, const char* clov, int block, cudaStream_t st) {
  const dim3 grid((unsigned)(a.nblk * a.nrhs));
  BR_PREC_SWITCH(prec, k_clover_site, a, clov)
}
bool launch_g5_site(int prec, const CopyArgs& a, const char* clov, int block, cudaStream_t st) {
  const dim3 grid((unsigned)(a.nblk * a.nrhs));
  BR_PREC_SWITCH(prec, k_g5_site, a, clov)
}

template <int PS>
static bool convert_to(int pd, const CopyArgs& a, int block, cudaStream_t st) {
  const dim3 grid((unsigned)(a.nblk * a.nrhs));
  switch (pd) {
    case P_F64: k_convert<PS, P_F64><<<grid, block, 0, st>>>(a); return true;
    case P_F32: k_convert<PS, P_F32><<<grid, block, 0, st>>>(a); return true;
    case P_F16: k_convert<PS, P_F16><<<grid, block, 0, st>>>(a); return true;
    case P_BF16: k_convert<PS, P_BF16><<<grid, block, 0, st>>>(a); return true;
  }
  return false;
}
bool launch_convert(int ps, int pd, const CopyArgs& a, int block, cudaStream_t st) {
  switch (ps) {
    case P_F64: return convert_to<P_F64>(pd, a, block, st);
    case P_F32: return convert_to<P_F32>(pd, a, block, st);
    case P_F16: return convert_to<P_F16>(pd, a, block, st);
    case P_BF16: return convert_to<P_BF16>(pd, a, block, st);
  }
  return false;
}

// ----------------------------------------------------------- gauge field
__global__ void __launch_bounds__(256) k_gauge_from_canon(const double* U, const Geom g, char* g64) {
  const long vh = g.vh, V = 2 * vh;
  const long lbb = link_block_bytes(P_F64, vh);
  const long n = 8 * vh;  // (parity, mu, ih)
  for (long k = (long)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (long)gridDim.x * blockDim.x) {
    const uint32_t ih = (uint32_t)(k % vh);
    const int mu = (int)((k / vh) % 4), p = (int)(k / (4 * vh));
    int c[4];
    uint32_t xh;
    site_coords(g, ih, p, c, xh);
    const long lex = 2 * (long)ih + (c[0] & 1);
    const double2* src = reinterpret_cast<const double2*>(U) + ((long)mu * V + lex) * 9;
    double2* dst = reinterpret_cast<double2*>(g64 + (long)(p * 4 + mu) * lbb);
#pragma unroll
    for (int e = 0; e < 9; ++e) dst[e * vh + ih] = __ldg(src + e);
  }
}

void launch_gauge_from_canon(const double* U, const Geom& g, char* g64, cudaStream_t st) {
  const long n = 8L * g.vh;
  const int block = 256;
  const long grid = (n + block - 1) / block;
  k_gauge_from_canon<<<(unsigned)(grid < 152 * 64 ? grid : 152 * 64), block, 0, st>>>(U, g, g64);
}

template <int P>
__global__ void __launch_bounds__(256) k_gauge_convert(const Geom g, const char* g64, char* gp) {
  const long vh = g.vh;
  const long l64 = link_block_bytes(P_F64, vh), lp = link_block_bytes(P, vh);
  const long n = 8 * vh;
  for (long k = (long)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (long)gridDim.x * blockDim.x) {
    const uint32_t ih = (uint32_t)(k % vh);
    const int blk = (int)(k / vh);  // parity * 4 + mu
    Link<double> u;
    load_link<P_F64>(g64 + blk * l64, vh, ih, u);
    char* base = gp + blk * lp;
    if constexpr (P == P_F32) {
      float4* d = reinterpret_cast<float4*>(base);
      d[ih] = make_float4((float)u.m[0][0].r, (float)u.m[0][0].i, (float)u.m[0][1].r, (float)u.m[0][1].i);
      d[vh + ih] = make_float4((float)u.m[0][2].r, (float)u.m[0][2].i, (float)u.m[1][0].r, (float)u.m[1][0].i);
      d[2 * vh + ih] = make_float4((float)u.m[1][1].r, (float)u.m[1][1].i, (float)u.m[1][2].r, (float)u.m[1][2].i);
    } else if constexpr (P == P_F16 || P == P_BF16) {
      H16<P> h;
      uint2* d = reinterpret_cast<uint2*>(base);
      auto w = [&](int r, int c) { return h.from2((float)u.m[r][c].r, (float)u.m[r][c].i); };
      d[ih] = make_uint2(w(0, 0), w(0, 1));
      d[vh + ih] = make_uint2(w(0, 2), w(1, 0));
      d[2 * vh + ih] = make_uint2(w(1, 1), w(1, 2));
    }
  }
}

bool launch_gauge_convert(int prec, const Geom& g, const char* g64, char* gp, cudaStream_t st) {
  const long n = 8L * g.vh;
  const int block = 256;
  long grid = (n + block - 1) / block;
  if (grid > 152 * 64) grid = 152 * 64;
  switch (prec) {
    case P_F32: k_gauge_convert<P_F32><<<(unsigned)grid, block, 0, st>>>(g, g64, gp); return true;
    case P_F16: k_gauge_convert<P_F16><<<(unsigned)grid, block, 0, st>>>(g, g64, gp); return true;
    case P_BF16: k_gauge_convert<P_BF16><<<(unsigned)grid, block, 0, st>>>(g, g64, gp); return true;
  }
  return false;
}

// ------------------------------------------------------------ clover term
template <int P>
__global__ void __launch_bounds__(256) k_clover_convert(const Geom g, const char* c64, char* cp) {
  const long vh = g.vh;
  const long b64 = clover_block_bytes(P_F64, vh), bp = clover_block_bytes(P, vh);
  const long n = 2 * vh;
  for (long k = (long)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (long)gridDim.x * blockDim.x) {
    const uint32_t ih = (uint32_t)(k % vh);
    const int p = (int)(k / vh);
    const double2* s = reinterpret_cast<const double2*>(c64 + p * b64);
    char* base = cp + p * bp;
    if constexpr (P == P_F32) {
      float4* d = reinterpret_cast<float4*>(base);
#pragma unroll
      for (int q = 0; q < 18; ++q) {
        double2 a = __ldg(s + (2 * q) * vh + ih), b = __ldg(s + (2 * q + 1) * vh + ih);
        d[q * vh + ih] = make_float4((float)a.x, (float)a.y, (float)b.x, (float)b.y);
      }
    } else {
      H16<P> h;
      uint32_t* d = reinterpret_cast<uint32_t*>(base);
#pragma unroll
      for (int w = 0; w < 36; ++w) {
        double2 a = __ldg(s + w * vh + ih);
        d[((w >> 2) * vh + ih) * 4 + (w & 3)] = h.from2((float)a.x, (float)a.y);
      }
    }
  }
}

bool launch_clover_convert(int prec, const Geom& g, const char* c64, char* cp, cudaStream_t st) {
  const long n = 2L * g.vh;
  const int block = 256;
  long grid = (n + block - 1) / block;
  if (grid > 152 * 64) grid = 152 * 64;
  switch (prec) {
    case P_F32: k_clover_convert<P_F32><<<(unsigned)grid, block, 0, st>>>(g, c64, cp); return true;
    case P_F16: k_clover_convert<P_F16><<<(unsigned)grid, block, 0, st>>>(g, c64, cp); return true;
    case P_BF16: k_clover_convert<P_BF16><<<(unsigned)grid, block, 0, st>>>(g, c64, cp); return true;
  }
  return false;
}

}  // namespace bridge
