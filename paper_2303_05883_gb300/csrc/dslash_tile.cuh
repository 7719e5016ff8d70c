// Multi-RHS hopping stencil with the link and clover work shared across the
// right-hand sides of a site (the paper solves O(10) equations on one gauge
// field, Sec. 3; Eq. 1 for the even-odd blocks).
//
// One block covers a tile of TILE_SITES consecutive output sites for a group
// of G <= TILE_MAX_RHS right-hand sides: blockDim = 32 G, warp w handles
// right-hand side (group start + w) for the 32 sites of the tile, so every
// spinor access of a warp is one coalesced 512-byte row per plane.  Per tile
// the block first stages, once for all G right-hand sides,
//   * the eight links of each site (row 2 rebuilt, the backward links stored
//     as their adjoint, every link pre-multiplied by beta and by the boundary
//     phase of its hop) as FP32 in shared memory,
//   * the T^-1 blocks of the site (F_E_CLOV), unpacked to FP32,
//   * the half-lattice indices of the eight neighbours,
// and then each thread runs the eight projected hops of its (site, rhs) with
// the link read from shared memory.  Compared with one independent thread
// per (site, rhs), the link loads, the 16-bit conversions of links and
// clover entries, the row-3 reconstruction, the neighbour arithmetic and the
// beta / phase multiplications are done once per site instead of once per
// right-hand side.
#pragma once

#include "dslash.cuh"

namespace bridge {

constexpr int TILE_SITES = 32;
constexpr int TILE_MAX_RHS = 12;
constexpr int TILE_THREADS = 32 * TILE_MAX_RHS;
// Staged per chunk of S = NT x 32 sites (NT tiles between two barriers), in
// float4 units: links [8 hops][5][S] (nine complex entries in five float4),
// clover [2 blocks][9][S], then the neighbour indices [8][S] as uint32.
// With pipelined neighbour loads (pf) each thread also owns two slots of
// four uint4 (three for the 16-bit spinor, one for its scale):
// [2 stages][4][TILE_THREADS] uint4.
BR_HD size_t tile_smem_bytes(bool clov, int nt, bool pf = false) {
  const int S = nt * TILE_SITES;
  return (size_t)(8 * 5 * S + (clov ? 2 * 9 * S : 0)) * 16 + (size_t)8 * S * 4 +
         (pf ? (size_t)2 * 4 * TILE_THREADS * 16 : 0);
}
// Right-hand sides per block for nrhs (groups of equal size, at most TILE_MAX_RHS).
BR_HD int tile_groups(int nrhs) { return (nrhs + TILE_MAX_RHS - 1) / TILE_MAX_RHS; }
BR_HD int tile_group_size(int nrhs) {
  const int ng = tile_groups(nrhs);
  return (nrhs + ng - 1) / ng;
}

// Reconstruction of the four-spin contribution of one hop from the two
// projected components u, each scaled by sc (the neighbour's per-site scale
// for 16-bit storage): the scale rides on the accumulation FMAs.
template <int MU, bool FWD>
BR_D void reconstruct_scaled(const cx<float> u[2][3], float sc, cx<float> acc[12]) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const cx<float> u0 = u[0][c], u1 = u[1][c];
    acc[c] = caxpy(sc, u0, acc[c]);
    acc[3 + c] = caxpy(sc, u1, acc[3 + c]);
    if (MU == 0) {
      acc[6 + c] = caxpy(sc, FWD ? times_mi(u1) : times_i(u1), acc[6 + c]);
      acc[9 + c] = caxpy(sc, FWD ? times_mi(u0) : times_i(u0), acc[9 + c]);
    } else if (MU == 1) {
      acc[6 + c] = caxpy(FWD ? -sc : sc, u1, acc[6 + c]);
      acc[9 + c] = caxpy(FWD ? sc : -sc, u0, acc[9 + c]);
    } else if (MU == 2) {
      acc[6 + c] = caxpy(sc, FWD ? times_mi(u0) : times_i(u0), acc[6 + c]);
      acc[9 + c] = caxpy(sc, FWD ? times_i(u1) : times_mi(u1), acc[9 + c]);
    } else {
      acc[6 + c] = caxpy(FWD ? -sc : sc, u0, acc[6 + c]);
      acc[9 + c] = caxpy(FWD ? -sc : sc, u1, acc[9 + c]);
    }
  }
}

// Spin projection of an FP16 spinor in packed half2 arithmetic (w[k]: the
// (re, im) pair of component k = spin * 3 + colour, unscaled), then widened
// to FP32: one add per complex pair instead of two FP32 adds after four
// conversions.  Multiplying by +-i swaps the pair and flips one sign.
template <int MU, bool FWD>
BR_D void project_f16(const uint32_t w[12], cx<float> hh[2][3]) {
  const __half2 ip = __floats2half2_rn(-1.0f, 1.0f);  // i (a, b) = swap(a, b) * (-1, +1)
  const __half2 im = __floats2half2_rn(1.0f, -1.0f);  // -i (a, b) = swap(a, b) * (+1, -1)
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const __half2 p0 = *reinterpret_cast<const __half2*>(&w[c]), p1 = *reinterpret_cast<const __half2*>(&w[3 + c]);
    const __half2 p2 = *reinterpret_cast<const __half2*>(&w[6 + c]), p3 = *reinterpret_cast<const __half2*>(&w[9 + c]);
    __half2 a, b;
    if (MU == 0) {
      a = __hfma2(__lowhigh2highlow(p3), FWD ? ip : im, p0);
      b = __hfma2(__lowhigh2highlow(p2), FWD ? ip : im, p1);
    } else if (MU == 1) {
      a = FWD ? __hadd2(p0, p3) : __hsub2(p0, p3);
      b = FWD ? __hsub2(p1, p2) : __hadd2(p1, p2);
    } else if (MU == 2) {
      a = __hfma2(__lowhigh2highlow(p2), FWD ? ip : im, p0);
      b = __hfma2(__lowhigh2highlow(p3), FWD ? im : ip, p1);
    } else {
      a = FWD ? __hsub2(p0, p2) : __hadd2(p0, p2);
      b = FWD ? __hsub2(p1, p3) : __hadd2(p1, p3);
    }
    const float2 fa = __half22float2(a), fb = __half22float2(b);
    hh[0][c] = {fa.x, fa.y};
    hh[1][c] = {fb.x, fb.y};
  }
}

// Stage the link of hop h (= 2 mu + backward) of chunk site s (S sites per chunk).
template <int P, int MU, int S>
BR_D void tile_stage_link(const HopArgs& a, const char* g_out, const char* g_in, long lbb, uint32_t ih, int p, int h,
                          int s, float4* sl, uint32_t* snb) {
  int c[4];
  uint32_t xh;
  site_coords(a.g, ih, p, c, xh);
  uint32_t f, b;
  bool wf, wb;
  neighbours<MU>(a.g, ih, c, xh, f, b, wf, wb);
  const bool fwd = (h & 1) == 0;
  Link<float> U;
  load_link<P, true>((fwd ? g_out : g_in) + MU * lbb, a.g.vh, fwd ? ih : b, U);
  const float coef = a.betaf * ((fwd ? wf : wb) ? a.bcf[MU] : 1.0f);
  cx<float> m[9];
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int q = 0; q < 3; ++q) m[3 * r + q] = fwd ? coef * U.m[r][q] : coef * conj(U.m[q][r]);
  float4* d = sl + h * 5 * S + s;
  d[0 * S] = make_float4(m[0].r, m[0].i, m[1].r, m[1].i);
  d[1 * S] = make_float4(m[2].r, m[2].i, m[3].r, m[3].i);
  d[2 * S] = make_float4(m[4].r, m[4].i, m[5].r, m[5].i);
  d[3 * S] = make_float4(m[6].r, m[6].i, m[7].r, m[7].i);
  d[4 * S] = make_float4(m[8].r, m[8].i, 0.f, 0.f);
  snb[h * S + s] = fwd ? f : b;
}

// One hop of one (site, rhs) with the staged link M (already beta * phase *
// U or its adjoint): acc += (1 -/+ gamma_mu) M psi(neighbour).
template <int P, int MU, bool FWD, int S>
BR_D void tile_hop(const char* in, long vh, const float4* sl, const uint32_t* snb, int s, cx<float> acc[12]) {
  constexpr int h = 2 * MU + (FWD ? 0 : 1);
  const uint32_t nb = snb[h * S + s];
  cx<float> hh[2][3];
  float sc = 1.0f;
  if constexpr (P == P_F16) {
    const uint4* pl = reinterpret_cast<const uint4*>(in);
    const uint4 v0 = __ldg(pl + nb), v1 = __ldg(pl + vh + nb), v2 = __ldg(pl + 2 * vh + nb);
    sc = __ldg(reinterpret_cast<const float*>(in + 48 * vh) + nb);
    const uint32_t w[12] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w, v2.x, v2.y, v2.z, v2.w};
    project_f16<MU, FWD>(w, hh);
  } else if constexpr (Tr<P>::half) {
    cx<float> psi[12];
    sc = load_spinor_unscaled<P>(in, vh, nb, psi);
    project<float, MU, FWD>(psi, hh);
  } else {
    cx<float> psi[12];
    load_spinor<P>(in, vh, nb, psi);
    project<float, MU, FWD>(psi, hh);
  }
  const float4* q = sl + h * 5 * S + s;
  const float4 q0 = q[0], q1 = q[S], q2 = q[2 * S], q3 = q[3 * S], q4 = q[4 * S];
  const cx<float> m00 = {q0.x, q0.y}, m01 = {q0.z, q0.w}, m02 = {q1.x, q1.y};
  const cx<float> m10 = {q1.z, q1.w}, m11 = {q2.x, q2.y}, m12 = {q2.z, q2.w};
  const cx<float> m20 = {q3.x, q3.y}, m21 = {q3.z, q3.w}, m22 = {q4.x, q4.y};
  cx<float> u[2][3];
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    u[k][0] = crow3(m00, m01, m02, hh[k]);
    u[k][1] = crow3(m10, m11, m12, hh[k]);
    u[k][2] = crow3(m20, m21, m22, hh[k]);
  }
  if constexpr (Tr<P>::half)
    reconstruct_scaled<MU, FWD>(u, sc, acc);
  else
    reconstruct<float, MU, FWD>(u, acc);
}

// Pipelined neighbour loads (16-bit storage): the neighbour spinor and scale
// of the next hop are copied into the thread's own shared-memory slot by
// cp.async while the current hop computes, so the load latency is hidden
// without holding the next hop's data in registers.  Each thread reads only
// the slot it filled itself, after waiting for its own copies: no barrier.
BR_D void cp_async16(uint32_t dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
BR_D void cp_async4(uint32_t dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(dst), "l"(src) : "memory");
}
BR_D void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
BR_D void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Slot k (0..2 spinor planes, 3 scale) of stage st of thread t.
BR_D uint4* tile_pf_slot(uint4* pf, int st, int k, int t) { return pf + (st * 4 + k) * TILE_THREADS + t; }

// Start the copy of the neighbour of hop H (16-bit spinor: three uint4 planes and the scale).
template <int H, int S>
BR_D void tile_fetch(const char* in, long vh, const uint32_t* snb, int s, uint4* pf, int t) {
  const uint32_t nb = snb[H * S + s];
  const uint4* pl = reinterpret_cast<const uint4*>(in);
#pragma unroll
  for (int k = 0; k < 3; ++k)
    cp_async16((uint32_t)__cvta_generic_to_shared(tile_pf_slot(pf, H & 1, k, t)), pl + k * vh + nb);
  cp_async4((uint32_t)__cvta_generic_to_shared(tile_pf_slot(pf, H & 1, 3, t)),
            reinterpret_cast<const float*>(in + 48 * vh) + nb);
  cp_async_commit();
}

// Hop H from the staged neighbour: projection, link product, reconstruction.
template <int P, int H, int S>
BR_D void tile_hop_staged(const float4* sl, int s, const uint4* pf, int t, cx<float> acc[12]) {
  constexpr int MU = H / 2;
  constexpr bool FWD = (H & 1) == 0;
  const uint4 v0 = *tile_pf_slot(const_cast<uint4*>(pf), H & 1, 0, t);
  const uint4 v1 = *tile_pf_slot(const_cast<uint4*>(pf), H & 1, 1, t);
  const uint4 v2 = *tile_pf_slot(const_cast<uint4*>(pf), H & 1, 2, t);
  const float sc = __uint_as_float(tile_pf_slot(const_cast<uint4*>(pf), H & 1, 3, t)->x);
  cx<float> hh[2][3];
  if constexpr (P == P_F16) {
    const uint32_t w[12] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w, v2.x, v2.y, v2.z, v2.w};
    project_f16<MU, FWD>(w, hh);
  } else {
    H16<P> h;
    const uint32_t w[12] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w, v2.x, v2.y, v2.z, v2.w};
    cx<float> psi[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      const float2 f = h.to2(w[k]);
      psi[k] = {f.x, f.y};
    }
    project<float, MU, FWD>(psi, hh);
  }
  const float4* q = sl + H * 5 * S + s;
  const float4 q0 = q[0], q1 = q[S], q2 = q[2 * S], q3 = q[3 * S], q4 = q[4 * S];
  const cx<float> m00 = {q0.x, q0.y}, m01 = {q0.z, q0.w}, m02 = {q1.x, q1.y};
  const cx<float> m10 = {q1.z, q1.w}, m11 = {q2.x, q2.y}, m12 = {q2.z, q2.w};
  const cx<float> m20 = {q3.x, q3.y}, m21 = {q3.z, q3.w}, m22 = {q4.x, q4.y};
  cx<float> u[2][3];
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    u[k][0] = crow3(m00, m01, m02, hh[k]);
    u[k][1] = crow3(m10, m11, m12, hh[k]);
    u[k][2] = crow3(m20, m21, m22, hh[k]);
  }
  reconstruct_scaled<MU, FWD>(u, sc, acc);
}

// One pipeline step: start hop H + 1's copy, wait for hop H's, compute hop H.
template <int P, int H, int S>
BR_D void tile_pf_step(const char* in, long vh, const float4* sl, const uint32_t* snb, int s, uint4* pf, int t,
                       cx<float> acc[12]) {
  if constexpr (H < 7) {
    tile_fetch<H + 1, S>(in, vh, snb, s, pf, t);
    cp_async_wait<1>();
  } else {
    cp_async_wait<0>();
  }
  tile_hop_staged<P, H, S>(sl, s, pf, t, acc);
}

// NT tiles (NT x 32 sites) are staged between two barriers; the register
// budget allows two resident 384-thread blocks per SM.  PF: pipelined
// neighbour loads (16-bit storage only).
template <int P, int FL, int RED, int NT, bool PF = false>
__global__ void __launch_bounds__(32 * TILE_MAX_RHS, 2) hop_kernel_tile(const HopArgs a) {
  static_assert(!PF || Tr<P>::half, "pipelined neighbour loads: 16-bit storage");
  static_assert(P != P_F64, "FP32 arithmetic kernels only");
  constexpr int S = NT * TILE_SITES;
  extern __shared__ float4 tile_smem[];
  float4* sl = tile_smem;
  float4* sc_clov = tile_smem + 8 * 5 * S;
  uint32_t* snb = reinterpret_cast<uint32_t*>(tile_smem + 8 * 5 * S + ((FL & F_E_CLOV) ? 2 * 9 * S : 0));
  uint4* pf = reinterpret_cast<uint4*>(snb + 8 * S);  // PF slots
  const int ng = tile_groups(a.nrhs), G = tile_group_size(a.nrhs);
  const int grp = blockIdx.x % ng;
  const int sb = blockIdx.x / ng;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int rhs = grp * G + w;  // warp-uniform
  const long vh = a.g.vh;
  constexpr int NV = RED == R_NORM ? 1 : RED == R_DOT_A ? 2 : 3;
  const bool live = rhs < a.nrhs && w < G && !rhs_finished(a.red, rhs);
  PartialSum<float> ps[NV];
  const int p = a.out_parity;
  const long lbb = link_block_bytes(P, vh), cbb = clover_block_bytes(P, vh);
  const char* g_out = a.gauge + (long)p * 4 * lbb;
  const char* g_in = a.gauge + (long)(1 - p) * 4 * lbb;
  const char* in = a.in + (long)rhs * a.in_rs;
  const uint32_t nchunks = (uint32_t)((vh + S - 1) / S);
  constexpr int nstage = 8 * S + ((FL & F_E_CLOV) ? 2 * S : 0);
  for (uint32_t chunk = sb; chunk < nchunks; chunk += (uint32_t)a.nblk) {
    const uint32_t base = chunk * S;
    __syncthreads();  // the previous chunk's reads of the staged data are done
    for (int j = threadIdx.x; j < nstage; j += blockDim.x) {
      const int s = j % S;
      const uint32_t ih = base + s;
      if (ih >= (uint32_t)vh) continue;
      if (j < 8 * S) {
        const int h = j / S;
        switch (h >> 1) {
          case 0: tile_stage_link<P, 0, S>(a, g_out, g_in, lbb, ih, p, h, s, sl, snb); break;
          case 1: tile_stage_link<P, 1, S>(a, g_out, g_in, lbb, ih, p, h, s, sl, snb); break;
          case 2: tile_stage_link<P, 2, S>(a, g_out, g_in, lbb, ih, p, h, s, sl, snb); break;
          default: tile_stage_link<P, 3, S>(a, g_out, g_in, lbb, ih, p, h, s, sl, snb); break;
        }
      } else if constexpr ((FL & F_E_CLOV) != 0) {
        const int b = (j - 8 * S) / S;
        float m[36];
        // constant block index in each branch keeps the unpacking in registers
        if (b == 0)
          load_clover_block<P, true>(a.clovE + p * cbb, vh, ih, 0, m);
        else
          load_clover_block<P, true>(a.clovE + p * cbb, vh, ih, 1, m);
        float4* d = sc_clov + b * 9 * S + s;
#pragma unroll
        for (int k = 0; k < 9; ++k) d[k * S] = make_float4(m[4 * k], m[4 * k + 1], m[4 * k + 2], m[4 * k + 3]);
      }
    }
    __syncthreads();
    if (!live) continue;
#pragma unroll 1
    for (int t = 0; t < NT; ++t) {
      const int s = t * TILE_SITES + lane;
      const uint32_t ih = base + s;
      if (ih >= (uint32_t)vh) break;
      cx<float> acc[12];
#pragma unroll
      for (int k = 0; k < 12; ++k) acc[k] = czero<float>();
      if constexpr (PF) {
        const int t = threadIdx.x;
        tile_fetch<0, S>(in, vh, snb, s, pf, t);
        tile_pf_step<P, 0, S>(in, vh, sl, snb, s, pf, t, acc);
        tile_pf_step<P, 1, S>(in, vh, sl, snb, s, pf, t, acc);
        tile_pf_step<P, 2, S>(in, vh, sl, snb, s, pf, t, acc);
        tile_pf_step<P, 3, S>(in, vh, sl, snb, s, pf, t, acc);
        tile_pf_step<P, 4, S>(in, vh, sl, snb, s, pf, t, acc);
        tile_pf_step<P, 5, S>(in, vh, sl, snb, s, pf, t, acc);
        tile_pf_step<P, 6, S>(in, vh, sl, snb, s, pf, t, acc);
        tile_pf_step<P, 7, S>(in, vh, sl, snb, s, pf, t, acc);
      } else {
        tile_hop<P, 0, true, S>(in, vh, sl, snb, s, acc);
        tile_hop<P, 0, false, S>(in, vh, sl, snb, s, acc);
        tile_hop<P, 1, true, S>(in, vh, sl, snb, s, acc);
        tile_hop<P, 1, false, S>(in, vh, sl, snb, s, acc);
        tile_hop<P, 2, true, S>(in, vh, sl, snb, s, acc);
        tile_hop<P, 2, false, S>(in, vh, sl, snb, s, acc);
        tile_hop<P, 3, true, S>(in, vh, sl, snb, s, acc);
        tile_hop<P, 3, false, S>(in, vh, sl, snb, s, acc);
      }
      cx<float> v[12];
      if constexpr ((FL & F_E_CLOV) != 0) {
#pragma unroll
        for (int b = 0; b < 2; ++b) {
          float m[36];
          const float4* q = sc_clov + b * 9 * S + s;
#pragma unroll
          for (int k = 0; k < 9; ++k) {
            const float4 t4 = q[k * S];
            m[4 * k] = t4.x;
            m[4 * k + 1] = t4.y;
            m[4 * k + 2] = t4.z;
            m[4 * k + 3] = t4.w;
          }
          hermitian6_apply<float>(m, acc + 6 * b, v + 6 * b);
        }
      } else {
#pragma unroll
        for (int k = 0; k < 12; ++k) v[k] = acc[k];
      }
      cx<float> sv[12];
      if constexpr ((FL & F_SELF) != 0) {
        load_spinor<P, true, true>(a.self + (long)rhs * a.self_rs, vh, ih, sv);
#pragma unroll
        for (int k = 0; k < 12; ++k) v[k] = caxpy(a.s1f, sv[k], v[k]);
      }
      store_spinor<P>(a.out + (long)rhs * a.out_rs, vh, ih, v);
      if constexpr (RED == R_NORM) {
        float n = 0.f;
#pragma unroll
        for (int k = 0; k < 12; ++k) n = fmaf(v[k].r, v[k].r, fmaf(v[k].i, v[k].i, n));
        ps[0].add(n);
      } else if constexpr (RED == R_DOT_A) {
        cx<float> wv[12];
        load_spinor<P, true, true>(a.avec + (long)rhs * a.avec_rs, vh, ih, wv);
        cx<float> d = czero<float>();
#pragma unroll
        for (int k = 0; k < 12; ++k) d = cfma_conj(wv[k], v[k], d);
        ps[0].add(d.r);
        ps[1].add(d.i);
      } else if constexpr (RED == R_TS) {
        cx<float> d = czero<float>();
        float n = 0.f;
#pragma unroll
        for (int k = 0; k < 12; ++k) {
          d = cfma_conj(v[k], sv[k], d);
          n = fmaf(v[k].r, v[k].r, fmaf(v[k].i, v[k].i, n));
        }
        ps[0].add(d.r);
        ps[1].add(d.i);
        ps[2].add(n);
      }
    }
  }
  if constexpr (RED != R_NONE) {
    // one warp per right-hand side: the warp's sum is the block's partial
    double rv[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      rv[k] = ps[k].value();
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) rv[k] += __shfl_xor_sync(0xffffffffu, rv[k], off);
    }
    if (lane == 0 && rhs < a.nrhs && w < G)
#pragma unroll
      for (int k = 0; k < NV; ++k) a.red.partials[((long)rhs * a.nblk + sb) * 4 + k] = rv[k];
    grid_finish<NV>(a.red, a.nblk, a.nrhs);
  }
}

}  // namespace bridge
