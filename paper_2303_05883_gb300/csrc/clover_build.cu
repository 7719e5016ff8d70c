// Clover (Sheikholeslami-Wohlert) site term and its inverse, in FP64.
//
// The paper implements the clover operator (Sec. 2) without printing it;
// the form built here is the standard one:
//   T(x) = 1 - kappa c_sw sum_{mu<nu} sigma_{mu nu} F_{mu nu}(x),
//   F_{mu nu} = (Q_{mu nu} - Q_{mu nu}^dagger) / (8 i), made traceless,
//   Q_{mu nu}(x) = the four plaquettes of the (mu, nu) plane with a corner
//   at x, each run counter-clockwise from x.
// In the chiral basis sigma_{mu nu} is block diagonal in spin, so T is two
// Hermitian 6x6 blocks per site.  With sigma_1..3 the Pauli matrices:
//   sigma_xy = -s3 (+) -s3, sigma_xz = s2 (+) s2, sigma_yz = -s1 (+) -s1,
//   sigma_xt = s1 (+) -s1, sigma_yt = s2 (+) -s2, sigma_zt = s3 (+) -s3,
// so block b is 1 - kappa c_sw [[C, A - iB], [A + iB, -C]] with
//   upper: A = F_xt - F_yz, B = F_xz + F_yt, C = F_zt - F_xy
//   lower: A = -F_yz - F_xt, B = F_xz - F_yt, C = -F_xy - F_zt.
// One thread builds both blocks of one site and inverts them by
// Gauss-Jordan elimination with partial pivoting (setup, run once per gauge
// field and kappa c_sw).
#include "kernels.h"

namespace bridge {

using M3 = Link<double>;
using Z = cx<double>;

__device__ __forceinline__ void mm(const M3& a, const M3& b, M3& c) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) c.m[i][j] = a.m[i][0] * b.m[0][j] + a.m[i][1] * b.m[1][j] + a.m[i][2] * b.m[2][j];
}
__device__ __forceinline__ void mm_dag(const M3& a, const M3& b, M3& c) {  // a b^dagger
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      c.m[i][j] = a.m[i][0] * conj(b.m[j][0]) + a.m[i][1] * conj(b.m[j][1]) + a.m[i][2] * conj(b.m[j][2]);
}
__device__ __forceinline__ void dag_m(const M3& a, const M3& b, M3& c) {  // a^dagger b
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) c.m[i][j] = cmul_conj(a.m[0][i], b.m[0][j]) + cmul_conj(a.m[1][i], b.m[1][j]) + cmul_conj(a.m[2][i], b.m[2][j]);
}

struct Site {
  int c[4];
};

__device__ __forceinline__ Site shifted(const Geom& g, Site s, int mu, int step) {
  int v = s.c[mu] + step;
  if (v < 0) v += g.L[mu];
  if (v >= g.L[mu]) v -= g.L[mu];
  s.c[mu] = v;
  return s;
}

__device__ __forceinline__ void link_at(const Geom& g, const char* g64, long lbb, Site s, int mu, M3& u) {
  const int par = (s.c[0] + s.c[1] + s.c[2] + s.c[3]) & 1;
  const uint32_t ih = (uint32_t)(s.c[0] >> 1) + g.Lxh * ((uint32_t)s.c[1] + (uint32_t)g.L[1] * ((uint32_t)s.c[2] + (uint32_t)g.L[2] * (uint32_t)s.c[3]));
  load_link<P_F64>(g64 + (long)(par * 4 + mu) * lbb, g.vh, ih, u);
}

// F_{mu nu}(x), traceless.
__device__ void field_strength(const Geom& g, const char* g64, long lbb, Site x, int mu, int nu, M3& F) {
  M3 Q, a, b, c, t;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) Q.m[i][j] = czero<double>();
  const Site xpm = shifted(g, x, mu, +1), xpn = shifted(g, x, nu, +1);
  const Site xmm = shifted(g, x, mu, -1), xmn = shifted(g, x, nu, -1);
  const Site xmm_pn = shifted(g, xmm, nu, +1), xmm_mn = shifted(g, xmm, nu, -1), xpm_mn = shifted(g, xpm, nu, -1);
  // leaf 1: U_mu(x) U_nu(x+mu) U_mu(x+nu)^dag U_nu(x)^dag
  link_at(g, g64, lbb, x, mu, a);
  link_at(g, g64, lbb, xpm, nu, b);
  mm(a, b, c);
  link_at(g, g64, lbb, xpn, mu, a);
  mm_dag(c, a, t);
  link_at(g, g64, lbb, x, nu, a);
  mm_dag(t, a, c);
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) Q.m[i][j] = Q.m[i][j] + c.m[i][j];
  // leaf 2: U_nu(x) U_mu(x-mu+nu)^dag U_nu(x-mu)^dag U_mu(x-mu)
  link_at(g, g64, lbb, x, nu, a);
  link_at(g, g64, lbb, xmm_pn, mu, b);
  mm_dag(a, b, c);
  link_at(g, g64, lbb, xmm, nu, a);
  mm_dag(c, a, t);
  link_at(g, g64, lbb, xmm, mu, a);
  mm(t, a, c);
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) Q.m[i][j] = Q.m[i][j] + c.m[i][j];
  // leaf 3: U_mu(x-mu)^dag U_nu(x-mu-nu)^dag U_mu(x-mu-nu) U_nu(x-nu)
  link_at(g, g64, lbb, xmm_mn, nu, a);
  link_at(g, g64, lbb, xmm, mu, b);
  mm(a, b, c);  // U_nu(x-mu-nu) U_mu(x-mu)
  // (U_mu(x-mu)^dag U_nu(x-mu-nu)^dag) = (U_nu(x-mu-nu) U_mu(x-mu))^dag
  link_at(g, g64, lbb, xmm_mn, mu, a);
  dag_m(c, a, t);
  link_at(g, g64, lbb, xmn, nu, a);
  mm(t, a, c);
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) Q.m[i][j] = Q.m[i][j] + c.m[i][j];
  // leaf 4: U_nu(x-nu)^dag U_mu(x-nu) U_nu(x+mu-nu) U_mu(x)^dag
  link_at(g, g64, lbb, xmn, nu, a);
  link_at(g, g64, lbb, xmn, mu, b);
  dag_m(a, b, c);
  link_at(g, g64, lbb, xpm_mn, nu, a);
  mm(c, a, t);
  link_at(g, g64, lbb, x, mu, a);
  mm_dag(t, a, c);
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) Q.m[i][j] = Q.m[i][j] + c.m[i][j];
  // F = (Q - Q^dag) / (8 i) = -i/8 (Q - Q^dag), then remove trace / 3
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      Z d = Q.m[i][j] - conj(Q.m[j][i]);
      F.m[i][j] = {d.i * 0.125, -d.r * 0.125};
    }
  Z tr = F.m[0][0] + F.m[1][1] + F.m[2][2];
  tr = {tr.r / 3.0, tr.i / 3.0};
#pragma unroll
  for (int i = 0; i < 3; ++i) F.m[i][i] = F.m[i][i] - tr;
}

// In-place inverse of a 6x6 complex matrix (Gauss-Jordan, partial pivoting).
__device__ void invert6(Z a[6][6], Z inv[6][6]) {
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 6; ++j) inv[i][j] = (i == j) ? Z{1.0, 0.0} : czero<double>();
  for (int col = 0; col < 6; ++col) {
    int piv = col;
    double best = a[col][col].r * a[col][col].r + a[col][col].i * a[col][col].i;
    for (int r = col + 1; r < 6; ++r) {
      double m = a[r][col].r * a[r][col].r + a[r][col].i * a[r][col].i;
      if (m > best) {
        best = m;
        piv = r;
      }
    }
    if (piv != col)
      for (int j = 0; j < 6; ++j) {
        Z t = a[col][j];
        a[col][j] = a[piv][j];
        a[piv][j] = t;
        t = inv[col][j];
        inv[col][j] = inv[piv][j];
        inv[piv][j] = t;
      }
    const Z d = a[col][col];
    const double n = d.r * d.r + d.i * d.i;
    const Z rcp = {d.r / n, -d.i / n};
    for (int j = 0; j < 6; ++j) {
      a[col][j] = a[col][j] * rcp;
      inv[col][j] = inv[col][j] * rcp;
    }
    for (int r = 0; r < 6; ++r) {
      if (r == col) continue;
      const Z f = a[r][col];
      for (int j = 0; j < 6; ++j) {
        a[r][j] = a[r][j] - f * a[col][j];
        inv[r][j] = inv[r][j] - f * inv[col][j];
      }
    }
  }
}

__device__ void pack6(const Z m[6][6], double2* dst, long vh, uint32_t ih, int b) {
  double v[36];
  for (int r = 0; r < 6; ++r) v[r] = m[r][r].r;
  int k = 0;
  for (int r = 1; r < 6; ++r)
    for (int c = 0; c < r; ++c) {
      v[6 + 2 * k] = m[r][c].r;
      v[6 + 2 * k + 1] = m[r][c].i;
      ++k;
    }
  for (int q = 0; q < 18; ++q) dst[(18 * b + q) * vh + ih] = make_double2(v[2 * q], v[2 * q + 1]);
}

__global__ void __launch_bounds__(128) k_clover_build(const Geom g, const char* g64, double kcsw, char* T64, char* Tinv64) {
  const long vh = g.vh;
  const long lbb = link_block_bytes(P_F64, vh), cbb = clover_block_bytes(P_F64, vh);
  for (long k = (long)blockIdx.x * blockDim.x + threadIdx.x; k < 2 * vh; k += (long)gridDim.x * blockDim.x) {
    const uint32_t ih = (uint32_t)(k % vh);
    const int p = (int)(k / vh);
    Site x;
    uint32_t xh;
    site_coords(g, ih, p, x.c, xh);
    // plane order: xy, xz, xt, yz, yt, zt
    M3 F[6];
    field_strength(g, g64, lbb, x, 0, 1, F[0]);
    field_strength(g, g64, lbb, x, 0, 2, F[1]);
    field_strength(g, g64, lbb, x, 0, 3, F[2]);
    field_strength(g, g64, lbb, x, 1, 2, F[3]);
    field_strength(g, g64, lbb, x, 1, 3, F[4]);
    field_strength(g, g64, lbb, x, 2, 3, F[5]);
    for (int b = 0; b < 2; ++b) {
      const double sgn = b == 0 ? 1.0 : -1.0;
      Z blk[6][6], inv[6][6];
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
          // upper: A = F_xt - F_yz, B = F_xz + F_yt, C = F_zt - F_xy
          // lower: A = -F_xt - F_yz, B = F_xz - F_yt, C = -F_zt - F_xy
          const Z A = sgn * F[2].m[i][j] - F[3].m[i][j];
          const Z B = F[1].m[i][j] + sgn * F[4].m[i][j];
          const Z C = sgn * F[5].m[i][j] - F[0].m[i][j];
          const Z iB = times_i(B);
          const double id = (i == j) ? 1.0 : 0.0;
          blk[i][j] = Z{id, 0.0} - kcsw * C;
          blk[i][3 + j] = czero<double>() - kcsw * (A - iB);
          blk[3 + i][j] = czero<double>() - kcsw * (A + iB);
          blk[3 + i][3 + j] = Z{id, 0.0} + kcsw * C;
        }
      pack6(blk, reinterpret_cast<double2*>(T64 + p * cbb), vh, ih, b);
      invert6(blk, inv);
      pack6(inv, reinterpret_cast<double2*>(Tinv64 + p * cbb), vh, ih, b);
    }
  }
}

void launch_clover_build(const Geom& g, const char* g64, double kcsw, char* T64, char* Tinv64, cudaStream_t st) {
  const long n = 2L * g.vh;
  const int block = 128;
  long grid = (n + block - 1) / block;
  if (grid > 152 * 32) grid = 152 * 32;
  k_clover_build<<<(unsigned)grid, block, 0, st>>>(g, g64, kcsw, T64, Tinv64);
}

}  // namespace bridge
