// Two-level multigrid kernels for the clover operator (Sec. 3 of the paper:
// a DD-alpha-AMG variant with an SAP smoother, coarse BiCGStab and an outer
// Flexible BiCGStab).
//
// Blocks (the SAP domains, which are also the aggregates) tile the lattice;
// an aggregate is one block and one chirality (spins 0, 1 / 2, 3).  A CTA
// works on one block: thread j <-> site j of the block in lexicographic
// order of the block-local coordinates.  Fine fields are the usual
// full-lattice FP32 fields (two parity blocks of SoA planes); coarse vectors
// are [coarse site][chirality][vector] complex floats; the coarse operator is
// [coarse site][9 couplings][column b][row a] complex floats with coupling 0
// the block itself and 1 + 2 mu / 2 + 2 mu the blocks at +mu / -mu.
#pragma once

#include "dslash.cuh"
#include "reduce.cuh"

namespace bridge {

struct MgGeom {
  Geom g;       // fine lattice
  int b[4];     // block extents
  int cd[4];    // blocks per direction (even)
  int bsites;   // sites per block
  int nblocks;  // coarse sites
};

// Fine site of block-local index j in block blk: parity, half-lattice index
// and coordinates.
BR_HD void mg_site(const MgGeom& m, int blk, int j, int c[4], int& parity, uint32_t& ih) {
  int bc[4];
  int r = blk;
  for (int k = 0; k < 4; ++k) {
    bc[k] = r % m.cd[k];
    r /= m.cd[k];
  }
  int q = j;
  for (int k = 0; k < 4; ++k) {
    c[k] = bc[k] * m.b[k] + q % m.b[k];
    q /= m.b[k];
  }
  const long lex = c[0] + (long)m.g.L[0] * (c[1] + (long)m.g.L[1] * (c[2] + (long)m.g.L[2] * c[3]));
  parity = (c[0] + c[1] + c[2] + c[3]) & 1;
  ih = (uint32_t)(lex >> 1);
}

BR_HD int mg_block_colour(const MgGeom& m, int blk) {
  int s = 0, r = blk;
  for (int k = 0; k < 4; ++k) {
    s += r % m.cd[k];
    r /= m.cd[k];
  }
  return s & 1;
}

// The k-th block of one colour (the grid covers that colour only): with an
// even number of blocks along x, every row of blocks (fixed y, z, t block
// coordinates) holds cd[0] / 2 of each colour.
BR_HD int mg_colour_block(const MgGeom& m, int colour, int k) {
  const int half = m.cd[0] / 2;
  const int R = k / half, bx2 = k % half;
  const int s = R % m.cd[1] + (R / m.cd[1]) % m.cd[2] + R / (m.cd[1] * m.cd[2]);
  return 2 * bx2 + ((s + colour) & 1) + m.cd[0] * R;
}

// Coarse neighbour of block blk at +mu (dir = +1) or -mu (dir = -1), periodic.
BR_HD int mg_block_nbr(const MgGeom& m, int blk, int mu, int dir) {
  int bc[4], r = blk;
  for (int k = 0; k < 4; ++k) {
    bc[k] = r % m.cd[k];
    r /= m.cd[k];
  }
  bc[mu] = (bc[mu] + dir + m.cd[mu]) % m.cd[mu];
  return bc[0] + m.cd[0] * (bc[1] + m.cd[1] * (bc[2] + m.cd[2] * bc[3]));
}

// Block sum of one complex float over the CTA into thread 0 (all threads).
BR_D cx<float> mg_block_sum(cx<float> v, float2* sh) {
  for (int off = 16; off > 0; off >>= 1) {
    v.r += __shfl_xor_sync(0xffffffffu, v.r, off);
    v.i += __shfl_xor_sync(0xffffffffu, v.i, off);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();
  if (lane == 0) sh[warp] = make_float2(v.r, v.i);
  __syncthreads();
  cx<float> s = czero<float>();
  if (threadIdx.x == 0)
    for (int w = 0; w < nw; ++w) s = s + cx<float>{sh[w].x, sh[w].y};
  return s;
}

// Block sum broadcast to every thread.
BR_D cx<float> mg_block_allsum(cx<float> v, float2* sh) {
  cx<float> s = mg_block_sum(v, sh);
  if (threadIdx.x == 0) sh[0] = make_float2(s.r, s.i);
  __syncthreads();
  s = {sh[0].x, sh[0].y};
  __syncthreads();
  return s;
}

struct MgTransferArgs {
  MgGeom m;
  int nv;
  const char* V;   // nv FP32 full fields (the orthonormal aggregate bases)
  long V_rs;       // bytes between them
  long field_block;  // bytes of one parity block of a full FP32 field
  const char* fine_in;  // restrict: fine input (full FP32 field)
  char* fine_out;       // prolong: fine output
  int add;              // prolong: out += P c instead of out = P c
  const float2* coarse_in;  // prolong input [nblocks][2][nv]
  float2* coarse_out;       // restrict output
};

// Restriction c = P^dag v: one CTA per block, one vector at a time.
__global__ void __launch_bounds__(1024) mg_restrict_kernel(const MgTransferArgs a) {
  __shared__ float2 sh[32];
  const int blk = blockIdx.x, j = threadIdx.x;
  const bool on = j < a.m.bsites;
  cx<float> v[12];
  int c[4], p = 0;
  uint32_t ih = 0;
  if (on) {
    mg_site(a.m, blk, j, c, p, ih);
    load_spinor<P_F32>(a.fine_in + p * a.field_block, a.m.g.vh, ih, v);
  }
  for (int i = 0; i < a.nv; ++i) {
    cx<float> d0 = czero<float>(), d1 = czero<float>();
    if (on) {
      cx<float> w[12];
      load_spinor<P_F32>(a.V + i * a.V_rs + p * a.field_block, a.m.g.vh, ih, w);
#pragma unroll
      for (int k = 0; k < 6; ++k) d0 = d0 + cmul_conj(w[k], v[k]);
#pragma unroll
      for (int k = 6; k < 12; ++k) d1 = d1 + cmul_conj(w[k], v[k]);
    }
    const cx<float> s0 = mg_block_sum(d0, sh);
    if (threadIdx.x == 0) a.coarse_out[((long)blk * 2 + 0) * a.nv + i] = make_float2(s0.r, s0.i);
    const cx<float> s1 = mg_block_sum(d1, sh);
    if (threadIdx.x == 0) a.coarse_out[((long)blk * 2 + 1) * a.nv + i] = make_float2(s1.r, s1.i);
  }
}

// Prolongation v (+)= P c: one CTA per block.
__global__ void __launch_bounds__(1024) mg_prolong_kernel(const MgTransferArgs a) {
  const int blk = blockIdx.x, j = threadIdx.x;
  if (j >= a.m.bsites) return;
  int c[4], p;
  uint32_t ih;
  mg_site(a.m, blk, j, c, p, ih);
  cx<float> out[12];
  if (a.add) {
    load_spinor<P_F32, false>(a.fine_out + p * a.field_block, a.m.g.vh, ih, out);
  } else {
#pragma unroll
    for (int k = 0; k < 12; ++k) out[k] = czero<float>();
  }
  const float2* cb = a.coarse_in + (long)blk * 2 * a.nv;
  for (int i = 0; i < a.nv; ++i) {
    cx<float> w[12];
    load_spinor<P_F32>(a.V + i * a.V_rs + p * a.field_block, a.m.g.vh, ih, w);
    const float2 c0 = cb[i], c1 = cb[a.nv + i];
#pragma unroll
    for (int k = 0; k < 6; ++k) out[k] = out[k] + w[k] * cx<float>{c0.x, c0.y};
#pragma unroll
    for (int k = 6; k < 12; ++k) out[k] = out[k] + w[k] * cx<float>{c1.x, c1.y};
  }
  store_spinor<P_F32>(a.fine_out + p * a.field_block, a.m.g.vh, ih, out);
}

// Modified Gram-Schmidt of the nv vectors on every aggregate, in place, in
// FP32 (the order of the vectors fixes the basis): one CTA per block,
// chirality by chirality.
__global__ void __launch_bounds__(1024) mg_orthonormalize_kernel(const MgTransferArgs a) {
  __shared__ float2 sh[32];
  const int blk = blockIdx.x, j = threadIdx.x;
  const bool on = j < a.m.bsites;
  int c[4], p = 0;
  uint32_t ih = 0;
  if (on) mg_site(a.m, blk, j, c, p, ih);
  char* V = const_cast<char*>(a.V);
  for (int chi = 0; chi < 2; ++chi) {
    const int k0 = 6 * chi;
    for (int i = 0; i < a.nv; ++i) {
      cx<float> vi[12];
      if (on) load_spinor<P_F32, false>(V + i * a.V_rs + p * a.field_block, a.m.g.vh, ih, vi);
      for (int jj = 0; jj < i; ++jj) {
        cx<float> d = czero<float>();
        cx<float> vj[12];
        if (on) {
          load_spinor<P_F32, false>(V + jj * a.V_rs + p * a.field_block, a.m.g.vh, ih, vj);
          for (int k = k0; k < k0 + 6; ++k) d = d + cmul_conj(vj[k], vi[k]);
        }
        d = mg_block_allsum(d, sh);
        if (on)
          for (int k = k0; k < k0 + 6; ++k) vi[k] = vi[k] - d * vj[k];
      }
      float n = 0.f;
      if (on)
        for (int k = k0; k < k0 + 6; ++k) n += vi[k].r * vi[k].r + vi[k].i * vi[k].i;
      const cx<float> nn = mg_block_allsum(cx<float>{n, 0.f}, sh);
      const float inv = nn.r > 0.f ? rsqrtf(nn.r) : 0.f;
      if (on) {
        // write back only this chirality's components
        cx<float> full[12];
        load_spinor<P_F32, false>(V + i * a.V_rs + p * a.field_block, a.m.g.vh, ih, full);
        for (int k = k0; k < k0 + 6; ++k) full[k] = inv * vi[k];
        store_spinor<P_F32>(V + i * a.V_rs + p * a.field_block, a.m.g.vh, ih, full);
      }
      __syncthreads();
    }
  }
}

// Setup probe: y = D_B w (mode 0: the block-local operator, hops that leave
// the block dropped) or the single hop -kappa (1 -+ gamma_mu) U ... w(x +- mu)
// restricted to hops that cross into the neighbouring block (mode 1 + 2 mu
// for +mu, 2 + 2 mu for -mu).  FP32, one CTA per block.
struct MgProbeArgs {
  MgGeom m;
  int mode;
  float kappa;
  float bcf[4];
  const char* w;  // full FP32 field
  char* y;
  long field_block;
  const char* gauge;  // FP32 links
  const char* clov;   // FP32 clover T (both parities), mode 0
};

template <int MU>
BR_D void mg_probe_dir(const MgProbeArgs& a, int c[4], int p, uint32_t ih, bool do_fwd, bool do_bwd, cx<float> acc[12]) {
  const Geom& g = a.m.g;
  const long lbb = link_block_bytes(P_F32, g.vh);
  const char* g_out = a.gauge + (long)p * 4 * lbb;
  const char* g_in = a.gauge + (long)(1 - p) * 4 * lbb;
  const char* in = a.w + (1 - p) * a.field_block;
  uint32_t xh = (uint32_t)(c[0] >> 1);
  uint32_t f, b;
  bool wf, wb;
  neighbours<MU>(g, ih, c, xh, f, b, wf, wb);
  if (do_fwd) hop_one<P_F32, MU, true, false>(in, g_out + MU * lbb, g.vh, f, ih, wf, a.bcf[MU], acc);
  if (do_bwd) hop_one<P_F32, MU, false, false>(in, g_in + MU * lbb, g.vh, b, b, wb, a.bcf[MU], acc);
}

__global__ void __launch_bounds__(1024) mg_probe_kernel(const MgProbeArgs a) {
  const int blk = blockIdx.x, j = threadIdx.x;
  if (j >= a.m.bsites) return;
  int c[4], p;
  uint32_t ih;
  mg_site(a.m, blk, j, c, p, ih);
  int lc[4], q = j;
  for (int k = 0; k < 4; ++k) {
    lc[k] = q % a.m.b[k];
    q /= a.m.b[k];
  }
  // which hops stay in the block (blocks are at most half the lattice, so a
  // hop that wraps always leaves its block)
  bool fin[4], bin[4];
  for (int k = 0; k < 4; ++k) {
    fin[k] = lc[k] + 1 < a.m.b[k];
    bin[k] = lc[k] > 0;
  }
  bool fsel[4], bsel[4];
  for (int k = 0; k < 4; ++k) {
    if (a.mode == 0) {
      fsel[k] = fin[k];
      bsel[k] = bin[k];
    } else {
      const int mu = (a.mode - 1) >> 1, dir = ((a.mode - 1) & 1) ? -1 : 1;
      fsel[k] = k == mu && dir > 0 && !fin[k];
      bsel[k] = k == mu && dir < 0 && !bin[k];
    }
  }
  cx<float> acc[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) acc[k] = czero<float>();
  mg_probe_dir<0>(a, c, p, ih, fsel[0], bsel[0], acc);
  mg_probe_dir<1>(a, c, p, ih, fsel[1], bsel[1], acc);
  mg_probe_dir<2>(a, c, p, ih, fsel[2], bsel[2], acc);
  mg_probe_dir<3>(a, c, p, ih, fsel[3], bsel[3], acc);
  cx<float> out[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) out[k] = (-a.kappa) * acc[k];
  if (a.mode == 0) {
    cx<float> wv[12], tw[12];
    load_spinor<P_F32>(a.w + p * a.field_block, a.m.g.vh, ih, wv);
    clover_apply<P_F32>(a.clov + p * clover_block_bytes(P_F32, a.m.g.vh), a.m.g.vh, ih, wv, tw);
#pragma unroll
    for (int k = 0; k < 12; ++k) out[k] = out[k] + tw[k];
  }
  store_spinor<P_F32>(a.y + p * a.field_block, a.m.g.vh, ih, out);
}

// Coarse operator application y = D_c x (or y = b - D_c x with b != null):
// thread (coarse site, row a); rows of one site in consecutive threads.
struct MgCoarseArgs {
  MgGeom m;
  int n2;  // 2 nv
  const float2* Dc;     // FP32 coarse operator
  const __half2* Dch;   // the same in FP16 (used when non-null)
  const int* nbr;       // [nblocks][9] coarse site of each coupling
  const float2* x;
  const float2* b;
  float2* y;
  const float2* rhat;  // MG_CR_ALPHA: <rhat, y> -> FIN_ALPHA
  RedArgs red;
  int* err;     // mg_coarse_tma_kernel: 1 if a tile copy did not arrive in time, 2 if the copies
                // still in flight then did not land within the drain's bound either
  int wait_polls;  // mg_coarse_tma_kernel: polls of each site-loop wait before it gives up
                   // (MG_WAIT_POLLS normally; 0 gives up at once, for tests of the error path)
  int stages;   // mg_coarse_tma_kernel: tile buffers in shared memory (2 .. 4)
  // mg_coarse_tma_kernel only: the coarse sites of one colour (parity 0 / 1,
  // -1 all sites), the couplings d0 .. d1 - 1 summed, and the vector of the
  // MG_CR_OMEGA dot <y, xin> (null: x).
  int parity, d0, d1;
  const float2* xin;
};

enum MgCoarseRed { MG_CR_NONE = 0, MG_CR_ALPHA = 1, MG_CR_OMEGA = 2 };

// ---- bulk async copies (TMA) into shared memory, completed on an mbarrier
BR_D uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
BR_D void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
BR_D void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
BR_D void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
// One thread: announce `bytes` on the barrier and start the copy of `bytes`
// (a multiple of 16, both addresses 16-byte aligned) from global memory.
BR_D void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  uint64_t state;
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 %0, [%1], %2;"
               : "=l"(state)
               : "r"(smem_u32(bar)), "r"(bytes)
               : "memory");
  (void)state;
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}
// Wait for the phase of the given parity to complete, giving up after about
// a second or max_polls polls (returns false then; max_polls = 0 gives up
// without polling).
constexpr int MG_WAIT_POLLS = 1 << 22;
BR_D bool mbar_wait(uint64_t* bar, uint32_t parity, int max_polls = MG_WAIT_POLLS) {
  uint64_t t0;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
  for (int it = 0; it < max_polls; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    if (ok) return true;
    if ((it & 255) == 255) {
      uint64_t t;
      asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
      if (t - t0 > 1000000000ull) return false;
    }
  }
  return false;
}

// y = D_c x (or b - D_c x); with a fused reduction for the coarse BiCGStab:
// MG_CR_ALPHA <rhat, y>, MG_CR_OMEGA (<y, x>, |y|^2).  Coarse sites of a
// converged solve (red.sc->done) are skipped.
// Row `row` of coarse site X: N2 > 0 fixes the row length at compile time
// (the column loop unrolls into independent loads); N2 = 0 reads it from a.
BR_D float2 coarse_entry(const float2* p) { return __ldg(p); }
BR_D float2 coarse_entry(const __half2* p) { return __half22float2(__ldg(p)); }

// Row lengths with compile-time kernels.  For them the FP16 copy of the
// coarse operator is stored in 16-byte tiles, entries (row, 4 g .. 4 g + 3)
// of coupling d of site X in word ((X * 9 + d) * (N2 / 4) + g) * N2 + row,
// and applied by mg_coarse_tma_kernel.
BR_HD bool mg_coarse_unrolled(int n2) { return n2 == 8 || n2 == 16 || n2 == 24 || n2 == 32 || n2 == 48; }

template <int N2, class E>
BR_D cx<float> coarse_row(const MgCoarseArgs& a, const E* Dc, int X, int row) {
  const int n2 = N2 > 0 ? N2 : a.n2;
  cx<float> s0 = czero<float>(), s1 = czero<float>();
  for (int d = 0; d < 9; ++d) {
    const int Y = __ldg(a.nbr + X * 9 + d);
    const E* M = Dc + ((long)X * 9 + d) * n2 * n2 + row;
    const float2* xv = a.x + (long)Y * n2;
    if constexpr (N2 > 0) {
#pragma unroll
      for (int col = 0; col < N2; col += 2) {
        const float2 m0 = coarse_entry(M + (long)col * N2), v0 = __ldg(xv + col);
        const float2 m1 = coarse_entry(M + (long)(col + 1) * N2), v1 = __ldg(xv + col + 1);
        s0 = cfma(cx<float>{m0.x, m0.y}, cx<float>{v0.x, v0.y}, s0);
        s1 = cfma(cx<float>{m1.x, m1.y}, cx<float>{v1.x, v1.y}, s1);
      }
    } else {
      for (int col = 0; col < n2; ++col) {
        const float2 m = coarse_entry(M + (long)col * n2), v = __ldg(xv + col);
        s0 = cfma(cx<float>{m.x, m.y}, cx<float>{v.x, v.y}, s0);
      }
    }
  }
  return s0 + s1;
}

template <int RED, int N2>
__global__ void __launch_bounds__(256) mg_coarse_kernel(const MgCoarseArgs a) {
  const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const int n2 = N2 > 0 ? N2 : a.n2;
  const bool skip = RED != MG_CR_NONE && a.red.sc != nullptr && a.red.sc[0].done != RUNNING;
  double rv[3] = {0.0, 0.0, 0.0};
  if (!skip && t < (long)a.m.nblocks * n2) {
    const int X = (int)(t / n2), row = (int)(t % n2);
    // the tiled FP16 copy of the unrolled row lengths goes to mg_coarse_tma_kernel
    cx<float> s;
    if constexpr (N2 > 0)
      s = coarse_row<N2>(a, a.Dc, X, row);
    else
      s = a.Dch ? coarse_row<N2>(a, a.Dch, X, row) : coarse_row<N2>(a, a.Dc, X, row);
    if (a.b) {
      const float2 bb = a.b[t];
      s = cx<float>{bb.x, bb.y} - s;
    }
    a.y[t] = make_float2(s.r, s.i);
    if (RED == MG_CR_ALPHA) {
      const float2 h = a.rhat[t];
      const cx<float> d = cmul_conj(cx<float>{h.x, h.y}, s);
      rv[0] = d.r;
      rv[1] = d.i;
    } else if (RED == MG_CR_OMEGA) {
      const float2 xv = a.x[t];
      const cx<float> d = cmul_conj(s, cx<float>{xv.x, xv.y});
      rv[0] = d.r;
      rv[1] = d.i;
      rv[2] = (double)s.r * s.r + (double)s.i * s.i;
    }
  }
  if (RED == MG_CR_ALPHA) reduce_finalize<2>(a.red, 0, blockIdx.x, gridDim.x, 1, rv);
  if (RED == MG_CR_OMEGA) reduce_finalize<3>(a.red, 0, blockIdx.x, gridDim.x, 1, rv);
}

// The same operator from the tiled FP16 copy, streamed by the bulk-copy
// engine: a persistent CTA walks its coarse sites (the k-th site of its
// share: k = blockIdx.x, + gridDim.x, ...); the 9 * N2 * N2 FP16 entries of
// a site are contiguous, so one bulk copy per site (of the couplings d0 ..
// d1 - 1) moves them into one of `stages` shared-memory buffers while the
// CTA computes on the previous ones.  Thread (d, row) forms the row sum of
// coupling d from shared memory against x at the coupled site (staged in
// shared memory, its loads issued one site ahead), and N2 threads add the
// couplings: y = sum, or y = b - sum.  With a colour (parity >= 0) only that
// colour's sites are visited, which with the even-odd tiles (slot 0 =
// A^-1, slots 1..8 = A^-1 times the hopping couplings) applies the pieces
// of the even-odd preconditioned coarse system.  Coarse sites of a
// converged solve (red.sc->done) are skipped.
template <int N2>
__host__ __device__ constexpr long mg_coarse_tile_bytes() { return 9L * (N2 / 4) * N2 * 16; }

template <int RED, int N2>
__global__ void __launch_bounds__(256) mg_coarse_tma_kernel(const MgCoarseArgs a) {
  static_assert(N2 % 4 == 0 && 9 * N2 <= 512, "tiled rows of at most 56 entries");
  constexpr int NG = N2 / 4;
  constexpr long TILE = mg_coarse_tile_bytes<N2>();
  extern __shared__ __align__(16) unsigned char dsm[];
  __shared__ __align__(8) uint64_t bar[4];
  __shared__ float2 xs[9 * N2];
  __shared__ float2 part[9 * N2];
  constexpr long CT = TILE / 9;  // bytes of one coupling
  const int tid = threadIdx.x, nt = blockDim.x;
  const int stages = a.stages;
  const bool skip = RED != MG_CR_NONE && a.red.sc != nullptr && a.red.sc[0].done != RUNNING;
  const int nsites = a.parity < 0 ? a.m.nblocks : a.m.nblocks / 2, first = blockIdx.x, step = gridDim.x;
  const int mine = (skip || first >= nsites) ? 0 : (nsites - first + step - 1) / step;
  const int d0 = a.d0, nd = a.d1 - a.d0;
  const uint32_t cbytes = (uint32_t)(nd * CT);
  auto site = [&](int k) { return a.parity < 0 ? k : mg_colour_block(a.m, a.parity, k); };
  const char* src = reinterpret_cast<const char*>(a.Dch) + d0 * CT;
  double rv[3] = {0.0, 0.0, 0.0};
  if (tid == 0) {
    for (int k = 0; k < stages; ++k) mbar_init(&bar[k], 1);
    mbar_fence_init();
  }
  __syncthreads();
  if (tid == 0)
    for (int k = 0; k < stages && k < mine; ++k) {
      const int X = site(first + k * step);
      bulk_load(dsm + k * TILE, src + (long)X * TILE, cbytes, &bar[k]);
    }
  // x at the coupled sites of the first site (two entries per thread at most)
  float2 xn[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
  auto load_x = [&](int X) {
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int i = tid + q * nt;
      if (i < nd * N2) {
        const int Y = __ldg(a.nbr + X * 9 + d0 + i / N2);
        xn[q] = __ldg(a.x + (long)Y * N2 + i % N2);
      }
    }
  };
  if (mine > 0) load_x(site(first));
  bool failed = false;
  int it = 0;
  for (; it < mine; ++it) {
    const int X = site(first + it * step), buf = it % stages;
#pragma unroll
    for (int q = 0; q < 2; ++q)
      if (tid + q * nt < nd * N2) xs[tid + q * nt] = xn[q];
    if (it + 1 < mine) load_x(site(first + (it + 1) * step));
    // operands of this site's epilogue, loaded before the wait
    float2 eb = make_float2(0.f, 0.f), ev = make_float2(0.f, 0.f);
    if (tid < N2) {
      const long t = (long)X * N2 + tid;
      if (a.b) eb = a.b[t];
      if (RED == MG_CR_ALPHA) ev = a.rhat[t];
      if (RED == MG_CR_OMEGA) ev = a.xin ? a.xin[t] : a.x[t];
    }
    const bool ok = mbar_wait(&bar[buf], (uint32_t)((it / stages) & 1), a.wait_polls);
    if (!__syncthreads_and(ok)) {
      failed = true;
      break;
    }
    const uint4* tile = reinterpret_cast<const uint4*>(dsm + buf * TILE);
    for (int p = tid; p < nd * N2; p += nt) {
      const int d = p / N2, row = p % N2;
      const float2* xv = xs + d * N2;
      cx<float> s0 = czero<float>(), s1 = czero<float>();
#pragma unroll
      for (int g = 0; g < NG; ++g) {
        const uint4 w = tile[(d * NG + g) * N2 + row];
        const float2 m0 = __half22float2(*reinterpret_cast<const __half2*>(&w.x));
        const float2 m1 = __half22float2(*reinterpret_cast<const __half2*>(&w.y));
        const float2 m2 = __half22float2(*reinterpret_cast<const __half2*>(&w.z));
        const float2 m3 = __half22float2(*reinterpret_cast<const __half2*>(&w.w));
        const float2 x0 = xv[4 * g], x1 = xv[4 * g + 1], x2 = xv[4 * g + 2], x3 = xv[4 * g + 3];
        s0 = cfma(cx<float>{m0.x, m0.y}, cx<float>{x0.x, x0.y}, s0);
        s1 = cfma(cx<float>{m1.x, m1.y}, cx<float>{x1.x, x1.y}, s1);
        s0 = cfma(cx<float>{m2.x, m2.y}, cx<float>{x2.x, x2.y}, s0);
        s1 = cfma(cx<float>{m3.x, m3.y}, cx<float>{x3.x, x3.y}, s1);
      }
      const cx<float> sum = s0 + s1;
      part[p] = make_float2(sum.r, sum.i);
    }
    __syncthreads();  // buffer `buf` and xs are free again
    if (tid == 0 && it + stages < mine) {
      fence_proxy_async_smem();
      bulk_load(dsm + buf * TILE, src + (long)site(first + (it + stages) * step) * TILE, cbytes, &bar[buf]);
    }
    if (tid < N2) {
      cx<float> sv = czero<float>();
      for (int d = 0; d < nd; ++d) sv = sv + cx<float>{part[d * N2 + tid].x, part[d * N2 + tid].y};
      const long t = (long)X * N2 + tid;
      if (a.b) sv = cx<float>{eb.x, eb.y} - sv;
      a.y[t] = make_float2(sv.r, sv.i);
      if (RED == MG_CR_ALPHA) {
        const cx<float> d = cmul_conj(cx<float>{ev.x, ev.y}, sv);
        rv[0] += d.r;
        rv[1] += d.i;
      } else if (RED == MG_CR_OMEGA) {
        const cx<float> d = cmul_conj(sv, cx<float>{ev.x, ev.y});
        rv[0] += d.r;
        rv[1] += d.i;
        rv[2] += (double)sv.r * sv.r + (double)sv.i * sv.i;
      }
    }
  }
  if (failed) {
    // Let the copies still in flight land before the CTA exits and its
    // shared memory is handed to another CTA: every copy this CTA issued is
    // waited for with the full bound.  Should that run out as well (the copy
    // engine stopped answering), the word says so and the host reports that
    // the context is no longer reliable.
    bool drained = true;
    for (int k = it; k < mine && k < it + stages; ++k)
      drained = mbar_wait(&bar[k % stages], (uint32_t)((k / stages) & 1)) && drained;
    if (tid == 0) atomicMax(a.err, drained ? 1 : 2);
  }
  if (RED == MG_CR_ALPHA) reduce_finalize<2>(a.red, 0, blockIdx.x, gridDim.x, 1, rv);
  if (RED == MG_CR_OMEGA) reduce_finalize<3>(a.red, 0, blockIdx.x, gridDim.x, 1, rv);
}

// ---- even-odd preconditioning of the coarse system (setup)
// With E / O the coarse sites of the two colours (every hopping coupling
// joins opposite colours), D_c = [[A_E, H_EO], [H_OE, A_O]] with A the
// self couplings; the even-odd system is
//   (1 - A_E^-1 H_EO A_O^-1 H_OE) e_E = A_E^-1 r_E - A_E^-1 H_EO A_O^-1 r_O,
//   e_O = A_O^-1 r_O - A_O^-1 H_OE e_E.
// Its tiles hold A_X^-1 in slot 0 and A_X^-1 times each hopping coupling in
// slots 1..8.

// A_X^-1 for every coarse site by Gauss-Jordan elimination with partial
// pivoting on [A | 1] in shared memory (row-major, n x 2n), one CTA per site.
// Dc and Ainv are column-major (entry (row, col) at col * n + row).
// A pivot whose magnitude is below 1e-6 of the largest entry of A_X (or not
// finite) marks A_X as numerically singular in FP32: *singular is set and
// the host falls back to the full coarse system.
__global__ void __launch_bounds__(256) mg_invert_self_kernel(const float2* Dc, float2* Ainv, int n, int* singular) {
  extern __shared__ __align__(16) unsigned char dsm_inv[];
  float2* M = reinterpret_cast<float2*>(dsm_inv);  // [n][2n]
  float2* f = M + 2L * n * n;                      // [n] elimination factors
  __shared__ int piv;
  __shared__ float amax2;
  const int X = blockIdx.x, tid = threadIdx.x, nt = blockDim.x, w = 2 * n;
  const float2* A = Dc + (long)X * 9 * n * n;  // coupling 0
  for (int i = tid; i < n * w; i += nt) {
    const int r = i / w, c = i % w;
    M[i] = c < n ? A[(long)c * n + r] : make_float2(c - n == r ? 1.f : 0.f, 0.f);
  }
  __syncthreads();
  if (tid == 0) {
    float m = 0.f;
    for (int i = 0; i < n * n; ++i) {
      const float2 v = M[(i / n) * w + i % n];
      m = fmaxf(m, v.x * v.x + v.y * v.y);
    }
    amax2 = m;
  }
  for (int k = 0; k < n; ++k) {
    if (tid == 0) {
      int best = k;
      float bv = -1.f;
      for (int r = k; r < n; ++r) {
        const float2 v = M[r * w + k];
        const float m2 = v.x * v.x + v.y * v.y;
        if (m2 > bv) {
          bv = m2;
          best = r;
        }
      }
      piv = best;
      if (!(bv > 1e-12f * amax2) || !isfinite(bv)) atomicExch(singular, 1);
    }
    __syncthreads();
    const int pr = piv;
    if (pr != k)
      for (int c = tid; c < w; c += nt) {
        const float2 t = M[k * w + c];
        M[k * w + c] = M[pr * w + c];
        M[pr * w + c] = t;
      }
    __syncthreads();
    const float2 pv = M[k * w + k];
    const float den = pv.x * pv.x + pv.y * pv.y;
    const cx<float> inv{pv.x / den, -pv.y / den};
    __syncthreads();  // every thread has the pivot before row k changes
    for (int c = tid; c < w; c += nt) {
      const cx<float> v = cx<float>{M[k * w + c].x, M[k * w + c].y} * inv;
      M[k * w + c] = make_float2(v.r, v.i);
    }
    __syncthreads();
    for (int r = tid; r < n; r += nt) f[r] = M[r * w + k];
    __syncthreads();
    for (int i = tid; i < n * w; i += nt) {
      const int r = i / w, c = i % w;
      if (r != k) {
        const cx<float> v = cx<float>{M[i].x, M[i].y} - cx<float>{f[r].x, f[r].y} * cx<float>{M[k * w + c].x, M[k * w + c].y};
        M[i] = make_float2(v.r, v.i);
      }
    }
    __syncthreads();
  }
  float2* out = Ainv + (long)X * n * n;
  for (int i = tid; i < n * n; i += nt) {
    const int c = i / n, r = i % n;
    out[i] = M[r * w + n + c];
  }
}

// Deo[X][0] = A_X^-1, Deo[X][d] = A_X^-1 Dc[X][d] for d = 1..8 (column-major
// n x n each); one CTA per coarse site, A_X^-1 in shared memory.
__global__ void __launch_bounds__(256) mg_premul_kernel(const float2* Dc, const float2* Ainv, float2* Deo, int n) {
  extern __shared__ __align__(16) unsigned char dsm_pm[];
  float2* sa = reinterpret_cast<float2*>(dsm_pm);
  const int X = blockIdx.x, tid = threadIdx.x, nt = blockDim.x, nn = n * n;
  for (int i = tid; i < nn; i += nt) sa[i] = Ainv[(long)X * nn + i];
  __syncthreads();
  float2* out = Deo + (long)X * 9 * nn;
  for (int i = tid; i < 9 * nn; i += nt) {
    const int d = i / nn, rem = i % nn, c = rem / n, r = rem % n;
    if (d == 0) {
      out[i] = sa[rem];
      continue;
    }
    const float2* Md = Dc + ((long)X * 9 + d) * nn + (long)c * n;  // column c of coupling d
    cx<float> acc = czero<float>();
    for (int k = 0; k < n; ++k) acc = cfma(cx<float>{sa[k * n + r].x, sa[k * n + r].y}, cx<float>{Md[k].x, Md[k].y}, acc);
    out[i] = make_float2(acc.r, acc.i);
  }
}

// Coarse BiCGStab vector steps with the scalars on the device (BiCGScalars,
// the finalizers of reduce.cuh): INIT x = 0, r = rhat = p = b, v = 0, |b|^2;
// S s = r - alpha v; XR x += alpha p + omega s, r = s - omega t, (<rhat, r>,
// |r|^2); P p = r + beta (p - omega v).
enum MgCBicgOp { MG_CB_INIT = 0, MG_CB_S = 1, MG_CB_XR = 2, MG_CB_P = 3 };
struct MgCBicgArgs {
  long n;
  float2 *x, *r, *rhat, *p, *v, *s, *t;
  const float2* b;
  RedArgs red;
};

// Grid-stride over the coarse vector (the grid is a couple of CTAs per SM,
// so the fused reductions combine few block partials); per-thread sums in
// compensated FP32.
template <int OP>
__global__ void __launch_bounds__(256) mg_cbicg_kernel(const MgCBicgArgs a) {
  const BiCGScalars* q = a.red.sc;
  const bool skip = OP != MG_CB_INIT && q->done != RUNNING;
  PartialSum<float> p0, p1, p2;
  auto c = [](float2 f) { return cx<float>{f.x, f.y}; };
  auto f2 = [](cx<float> v) { return make_float2(v.r, v.i); };
  const cx<float> al{(float)q->alpha_r, (float)q->alpha_i}, om{(float)q->omega_r, (float)q->omega_i};
  const cx<float> be{(float)q->beta_r, (float)q->beta_i};
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; !skip && i < a.n; i += (long)gridDim.x * blockDim.x) {
    if (OP == MG_CB_INIT) {
      const float2 bb = a.b[i];
      a.x[i] = make_float2(0.f, 0.f);
      a.r[i] = bb;
      a.rhat[i] = bb;
      a.p[i] = bb;
      a.v[i] = make_float2(0.f, 0.f);
      p0.add(fmaf(bb.x, bb.x, bb.y * bb.y));
    } else if (OP == MG_CB_S) {
      a.s[i] = f2(c(a.r[i]) - al * c(a.v[i]));
    } else if (OP == MG_CB_XR) {
      const cx<float> sv = c(a.s[i]);
      a.x[i] = f2(c(a.x[i]) + al * c(a.p[i]) + om * sv);
      const cx<float> rn = sv - om * c(a.t[i]);
      a.r[i] = f2(rn);
      const cx<float> d = cmul_conj(c(a.rhat[i]), rn);
      p0.add(d.r);
      p1.add(d.i);
      p2.add(fmaf(rn.r, rn.r, rn.i * rn.i));
    } else {
      a.p[i] = f2(c(a.r[i]) + be * (c(a.p[i]) - om * c(a.v[i])));
    }
  }
  double rv[3] = {p0.value(), p1.value(), p2.value()};
  if (OP == MG_CB_INIT) reduce_finalize<1>(a.red, 0, blockIdx.x, gridDim.x, 1, rv);
  if (OP == MG_CB_XR) reduce_finalize<3>(a.red, 0, blockIdx.x, gridDim.x, 1, rv);
}

// SAP block solve: `steps` minimal-residual steps on D_B e = r_B for every
// block of one colour, then x_B += e.  One CTA per block (blocks of the other
// colour return at once); rho in shared memory, q and e in registers.
struct MgSapArgs {
  MgGeom m;
  int colour, steps;
  float kappa;
  const char* r;  // full FP32 field: the current residual, or with `fused` the right-hand side
  char* x;        // full FP32 field, updated
  long field_block;
  const char* gauge;
  const char* clov;
  int fused;      // 1: the block residual r - D x is formed at the start of the sweep
  float bcf[4];   // boundary phases (fused residual)
};

// The two hops of direction MU of the full operator at one site (x of the
// opposite parity in `in`), added to acc: the fused residual of the SAP sweep.
template <int MU>
BR_D void mg_sap_hops(const MgSapArgs& a, const char* in, const char* g_out, const char* g_in, long lbb, uint32_t ih,
                      const int c[4], cx<float> acc[12]) {
  uint32_t f, b;
  bool wf, wb;
  neighbours<MU>(a.m.g, ih, c, (uint32_t)c[0] >> 1, f, b, wf, wb);
  hop_one<P_F32, MU, true, false>(in, g_out + MU * lbb, a.m.g.vh, f, ih, wf, a.bcf[MU], acc);
  hop_one<P_F32, MU, false, false>(in, g_in + MU * lbb, a.m.g.vh, b, b, wb, a.bcf[MU], acc);
}

// Dynamic shared memory of mg_sap_kernel: rho, the 4 forward links (all 18
// reals) and, with CS, the clover term (72 reals) of every site of the block.
BR_HD long mg_sap_smem(int bsites, bool cs) { return (long)bsites * (12 * 8 + 4 * 18 * 4 + (cs ? 72 * 4 : 0)); }

// One SAP half sweep: every block of one colour solves D_B e = r_B by
// `steps` MR steps from e = 0 and adds e to x.  One CTA per block, one
// thread per site.  With `fused` the kernel first forms the residual
// r_B = b - D x at its own sites (full operator, all eight hops): x inside
// the block is changed only by this CTA, after that, and every site outside
// the block that a hop reaches belongs to a block of the other colour, which
// this sweep does not touch -- so no separate residual pass is needed.  The links of the block are staged in shared memory once,
// so the MR steps read them there: a hop inside the block in -mu uses
// U_mu(x - mu), the forward link of the neighbour site.  CS: the clover term
// is staged as well (up to 168 KB, one CTA per SM); otherwise each step
// reads it from L2 (up to 96 KB, two CTAs per SM).  The faster variant is
// picked by timing at setup.
template <bool CS>
__global__ void __launch_bounds__(256, CS ? 1 : 2) mg_sap_kernel(const MgSapArgs a) {
  extern __shared__ __align__(16) unsigned char dsm[];
  __shared__ float2 sh[32];
  const int blk = mg_colour_block(a.m, a.colour, blockIdx.x);
  const int j = threadIdx.x, nsite = a.m.bsites;
  const bool on = j < nsite;
  cx<float>* rho = reinterpret_cast<cx<float>*>(dsm);            // [12][nsite]
  float* lk = reinterpret_cast<float*>(rho + 12L * nsite);        // [4 mu][18][nsite]
  float* cl = lk + 72L * nsite;                                   // [72][nsite]
  const long vh = a.m.g.vh;
  const long lbb = link_block_bytes(P_F32, vh);
  int c[4], p = 0;
  uint32_t ih = 0;
  int nbf[4], nbb[4];  // block-local neighbours (-1 outside)
  cx<float> e[12];
  if (on) {
    mg_site(a.m, blk, j, c, p, ih);
    int q = j, stride = 1;
    for (int k = 0; k < 4; ++k) {
      const int lc = q % a.m.b[k];
      q /= a.m.b[k];
      nbf[k] = lc + 1 < a.m.b[k] ? j + stride : -1;
      nbb[k] = lc > 0 ? j - stride : -1;
      stride *= a.m.b[k];
    }
    cx<float> rr[12];
    load_spinor<P_F32>(a.r + p * a.field_block, vh, ih, rr);
    const char* g_out = a.gauge + (long)p * 4 * lbb;
    if (a.fused) {
      // rr = b - T x + kappa H x at this site
      const char* xin = a.x + (1 - p) * a.field_block;
      const char* g_in = a.gauge + (long)(1 - p) * 4 * lbb;
      cx<float> hx[12];
#pragma unroll
      for (int k = 0; k < 12; ++k) hx[k] = czero<float>();
      mg_sap_hops<0>(a, xin, g_out, g_in, lbb, ih, c, hx);
      mg_sap_hops<1>(a, xin, g_out, g_in, lbb, ih, c, hx);
      mg_sap_hops<2>(a, xin, g_out, g_in, lbb, ih, c, hx);
      mg_sap_hops<3>(a, xin, g_out, g_in, lbb, ih, c, hx);
      cx<float> xs[12], tx[12];
      load_spinor<P_F32>(a.x + p * a.field_block, vh, ih, xs);
      clover_apply<P_F32>(a.clov + p * clover_block_bytes(P_F32, vh), vh, ih, xs, tx);
#pragma unroll
      for (int k = 0; k < 12; ++k) rr[k] = caxpy(a.kappa, hx[k], rr[k] - tx[k]);
    }
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      rho[k * nsite + j] = rr[k];
      e[k] = czero<float>();
    }
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
      if (nbf[mu] < 0) continue;  // no hop of the block uses it
      Link<float> U;
      load_link<P_F32, true>(g_out + mu * lbb, vh, ih, U);
#pragma unroll
      for (int k = 0; k < 9; ++k) {
        lk[(mu * 18 + 2 * k) * nsite + j] = U.m[k / 3][k % 3].r;
        lk[(mu * 18 + 2 * k + 1) * nsite + j] = U.m[k / 3][k % 3].i;
      }
    }
    if (CS) {
      const char* clov = a.clov + p * clover_block_bytes(P_F32, vh);
#pragma unroll
      for (int b = 0; b < 2; ++b) {
        float t[36];
        load_clover_block<P_F32, true>(clov, vh, ih, b, t);
#pragma unroll
        for (int k = 0; k < 36; ++k) cl[(36 * b + k) * nsite + j] = t[k];
      }
    }
  }
  __syncthreads();
  const char* clov = a.clov + p * clover_block_bytes(P_F32, vh);
  for (int step = 0; step < a.steps; ++step) {
    cx<float> qv[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) qv[k] = czero<float>();
    if (on) {
      // H_B rho: hops to neighbours inside the block, all operands in shared memory
      cx<float> acc[12];
#pragma unroll
      for (int k = 0; k < 12; ++k) acc[k] = czero<float>();
#pragma unroll
      for (int mu = 0; mu < 4; ++mu) {
#pragma unroll
        for (int fb = 0; fb < 2; ++fb) {
          const int nb = fb == 0 ? nbf[mu] : nbb[mu];
          if (nb < 0) continue;
          cx<float> psi[12], h[2][3], u[2][3];
#pragma unroll
          for (int k = 0; k < 12; ++k) psi[k] = rho[k * nsite + nb];
          const float* lu = lk + (long)mu * 18 * nsite + (fb == 0 ? j : nb);
          Link<float> U;
#pragma unroll
          for (int k = 0; k < 9; ++k) U.m[k / 3][k % 3] = cx<float>{lu[(2 * k) * nsite], lu[(2 * k + 1) * nsite]};
          switch (mu * 2 + fb) {
            case 0: project<float, 0, true>(psi, h); break;
            case 1: project<float, 0, false>(psi, h); break;
            case 2: project<float, 1, true>(psi, h); break;
            case 3: project<float, 1, false>(psi, h); break;
            case 4: project<float, 2, true>(psi, h); break;
            case 5: project<float, 2, false>(psi, h); break;
            case 6: project<float, 3, true>(psi, h); break;
            default: project<float, 3, false>(psi, h); break;
          }
#pragma unroll
          for (int s = 0; s < 2; ++s)
#pragma unroll
            for (int r = 0; r < 3; ++r) {
              if (fb == 0)
                u[s][r] = crow3(U.m[r][0], U.m[r][1], U.m[r][2], h[s]);
              else
                u[s][r] = crow3_conj(U.m[0][r], U.m[1][r], U.m[2][r], h[s]);
            }
          switch (mu * 2 + fb) {
            case 0: reconstruct<float, 0, true>(u, acc); break;
            case 1: reconstruct<float, 0, false>(u, acc); break;
            case 2: reconstruct<float, 1, true>(u, acc); break;
            case 3: reconstruct<float, 1, false>(u, acc); break;
            case 4: reconstruct<float, 2, true>(u, acc); break;
            case 5: reconstruct<float, 2, false>(u, acc); break;
            case 6: reconstruct<float, 3, true>(u, acc); break;
            default: reconstruct<float, 3, false>(u, acc); break;
          }
        }
      }
      cx<float> mine[12], tr[12];
#pragma unroll
      for (int k = 0; k < 12; ++k) mine[k] = rho[k * nsite + j];
      if (CS) {
#pragma unroll
        for (int b = 0; b < 2; ++b) {
          float t[36];
#pragma unroll
          for (int k = 0; k < 36; ++k) t[k] = cl[(36 * b + k) * nsite + j];
          hermitian6_apply<float>(t, mine + 6 * b, tr + 6 * b);
        }
      } else {
        clover_apply<P_F32>(clov, vh, ih, mine, tr);
      }
#pragma unroll
      for (int k = 0; k < 12; ++k) qv[k] = caxpy(-a.kappa, acc[k], tr[k]);
    }
    // alpha = <q, rho> / <q, q> over the block
    cx<float> dqr = czero<float>();
    float dqq = 0.f;
    if (on) {
#pragma unroll
      for (int k = 0; k < 12; ++k) {
        const cx<float> rk = rho[k * nsite + j];
        dqr = cfma_conj(qv[k], rk, dqr);
        dqq = fmaf(qv[k].r, qv[k].r, fmaf(qv[k].i, qv[k].i, dqq));
      }
    }
    const cx<float> sqr = mg_block_allsum(dqr, sh);
    const cx<float> sqq = mg_block_allsum(cx<float>{dqq, 0.f}, sh);
    const cx<float> alpha = sqq.r > 0.f ? (1.f / sqq.r) * sqr : czero<float>();
    if (on) {
#pragma unroll
      for (int k = 0; k < 12; ++k) {
        const cx<float> rk = rho[k * nsite + j];
        e[k] = cfma(alpha, rk, e[k]);
        rho[k * nsite + j] = cfma(cx<float>{-alpha.r, -alpha.i}, qv[k], rk);
      }
    }
    __syncthreads();
  }
  if (on) {
    cx<float> xv[12];
    load_spinor<P_F32, false>(a.x + p * a.field_block, vh, ih, xv);
#pragma unroll
    for (int k = 0; k < 12; ++k) xv[k] = xv[k] + e[k];
    store_spinor<P_F32>(a.x + p * a.field_block, vh, ih, xv);
  }
}

// ------------------------------------------------------- flat vector kernels
// y = a x + b y + c z over n complex numbers (b == 0: y is not read; z may be
// null when c == 0), with T float2 or double2; and <x, y> partial sums.
template <class T, class S>
__global__ void __launch_bounds__(256) mg_axpbypcz_kernel(long n, cx<S> ca, const T* x, cx<S> cb, T* y, cx<S> cc,
                                                         const T* z) {
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const T xv = x[i];
    cx<S> v = ca * cx<S>{xv.x, xv.y};
    if (cb.r != S(0) || cb.i != S(0)) {
      const T yv = y[i];
      v = v + cb * cx<S>{yv.x, yv.y};
    }
    if (z) {
      const T zv = z[i];
      v = v + cc * cx<S>{zv.x, zv.y};
    }
    T o;
    o.x = v.r;
    o.y = v.i;
    y[i] = o;
  }
}

template <class T>
__global__ void __launch_bounds__(256) mg_dot_kernel(long n, const T* x, const T* y, double2* partial) {
  __shared__ double sr[8], si[8];
  using R = decltype(T{}.x);
  PartialSum<R> pr, pi;  // compensated FP32 sums for FP32 data: no FP64 instruction in the loop
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const T a = x[i], b = y[i];
    pr.add(fmar<R>(a.x, b.x, a.y * b.y));
    pi.add(fmar<R>(a.x, b.y, -a.y * b.x));
  }
  double ar = pr.value(), ai = pi.value();
  for (int off = 16; off > 0; off >>= 1) {
    ar += __shfl_xor_sync(0xffffffffu, ar, off);
    ai += __shfl_xor_sync(0xffffffffu, ai, off);
  }
  if ((threadIdx.x & 31) == 0) {
    sr[threadIdx.x >> 5] = ar;
    si[threadIdx.x >> 5] = ai;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double tr = 0, ti = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      tr += sr[w];
      ti += si[w];
    }
    partial[blockIdx.x] = make_double2(tr, ti);
  }
}

}  // namespace bridge
