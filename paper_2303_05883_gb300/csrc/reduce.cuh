// Deterministic grid reductions fused into the producing kernel, and the
// device-side BiCGStab scalar updates they feed.
//
// Each block reduces its per-thread partial sums (FP64) with a fixed
// shuffle tree, writes one partial per block, and the last block to finish
// (atomic ticket, no waiting) sums all partials in a fixed order and runs a
// finalizer.  The result is bit-reproducible for a given launch shape, which
// is what makes a solve give the same answer alone and in a mix of requests.
#pragma once

#include "common.cuh"

namespace bridge {

enum FinMode {
  FIN_NONE = 0,
  FIN_STORE = 1,
  FIN_ALPHA = 2,
  FIN_OMEGA = 3,
  FIN_RHO = 4,
  FIN_INIT = 5,
  FIN_CG_INIT = 6,   // s[0] = |b|^2 of the CG system
  FIN_CG_ALPHA = 7,  // s[0] = |D p|^2
  FIN_CG_BETA = 8    // s[0] = |r|^2 after the update
};

struct RedArgs {
  double* partials = nullptr;       // [nrhs][nblk][4]
  unsigned int* counter = nullptr;  // one ticket counter per launch site, reset by the last block
  BiCGScalars* sc = nullptr;        // per right-hand side (may be null)
  CGScalars* cg = nullptr;          // per right-hand side, CG finalizers (may be null)
  double* result = nullptr;         // [nrhs][4] for FIN_STORE
  int fin = FIN_NONE;               // FinMode
  int check_done = 0;               // blocks of a right-hand side whose solve has ended skip their work
};

// Complex helpers on the scalar struct (FP64, one thread).
struct zc {
  double r, i;
};
__device__ __forceinline__ zc zmul(zc a, zc b) { return {a.r * b.r - a.i * b.i, a.r * b.i + a.i * b.r}; }
__device__ __forceinline__ zc zdiv(zc a, zc b) {
  double d = b.r * b.r + b.i * b.i;
  return {(a.r * b.r + a.i * b.i) / d, (a.i * b.r - a.r * b.i) / d};
}
__device__ __forceinline__ double zabs2(zc a) { return a.r * a.r + a.i * a.i; }

// BiCGStab (van der Vorst 1992; the solver of Sec. 3) scalar recurrences.
__device__ inline void finalize(const RedArgs& ra, int rhs, const double s[4]) {
  BiCGScalars* q = ra.sc ? ra.sc + rhs : nullptr;
  switch (ra.fin) {
    case FIN_STORE:
#pragma unroll
      for (int k = 0; k < 4; ++k) ra.result[rhs * 4 + k] = s[k];
      break;
    case FIN_INIT: {  // s[0] = |b|^2 ; x = 0, r = rhat = p = b
      q->b2 = s[0];
      q->r2 = s[0];
      q->rhat2 = s[0];
      q->rho_r = s[0];
      q->rho_i = 0.0;
      q->alpha_r = q->omega_r = 1.0;
      q->alpha_i = q->omega_i = 0.0;
      q->beta_r = q->beta_i = 0.0;
      q->iter = 0;
      q->tol2 = q->tol2 * s[0];  // tol^2 was staged in tol2 by the host
      q->done = (s[0] == 0.0 || s[0] <= q->tol2) ? CONVERGED : RUNNING;
      break;
    }
    case FIN_ALPHA: {  // s = <rhat, v>
      if (q->done) break;
      zc rv = {s[0], s[1]};
      if (!(zabs2(rv) > 0.0) || !isfinite(s[0]) || !isfinite(s[1])) {
        q->done = BREAKDOWN;
        break;
      }
      zc a = zdiv(zc{q->rho_r, q->rho_i}, rv);
      q->alpha_r = a.r;
      q->alpha_i = a.i;
      break;
    }
    case FIN_OMEGA: {  // s = <t, s>, |t|^2
      if (q->done) break;
      if (s[2] > 0.0) {
        q->omega_r = s[0] / s[2];
        q->omega_i = s[1] / s[2];
      } else {
        q->omega_r = q->omega_i = 0.0;
      }
      break;
    }
    case FIN_RHO: {  // s = <rhat, r>, |r|^2 after x, r were updated
      if (q->done) break;
      q->iter += 1;
      q->r2 = s[2];
      zc rho_new = {s[0], s[1]};
      if (!isfinite(s[2])) {
        q->done = BREAKDOWN;
      } else if (s[2] <= q->tol2) {
        q->done = CONVERGED;
      } else if (q->omega_r == 0.0 && q->omega_i == 0.0) {
        q->done = BREAKDOWN;
      } else if (zabs2(rho_new) < 1e-60 * q->rhat2 * s[2]) {
        q->done = BREAKDOWN;
      } else {
        zc b = zmul(zdiv(rho_new, zc{q->rho_r, q->rho_i}), zdiv(zc{q->alpha_r, q->alpha_i}, zc{q->omega_r, q->omega_i}));
        q->beta_r = b.r;
        q->beta_i = b.i;
        q->rho_r = rho_new.r;
        q->rho_i = rho_new.i;
        if (q->iter >= q->max_iter) q->done = MAXITER;
      }
      break;
    }
    case FIN_CG_INIT: {  // r = p = b, x = 0
      CGScalars* g = ra.cg + rhs;
      g->b2 = s[0];
      g->rr = s[0];
      g->alpha = g->beta = 0.0;
      g->iter = 0;
      g->tol2 = g->tol2 * s[0];
      g->done = !isfinite(s[0]) ? BREAKDOWN : (s[0] == 0.0 || s[0] <= g->tol2) ? CONVERGED : RUNNING;
      break;
    }
    case FIN_CG_ALPHA: {
      CGScalars* g = ra.cg + rhs;
      if (g->done) break;
      g->pq = s[0];
      if (!(s[0] > 0.0) || !isfinite(s[0]))
        g->done = BREAKDOWN;
      else
        g->alpha = g->rr / s[0];
      break;
    }
    case FIN_CG_BETA: {
      CGScalars* g = ra.cg + rhs;
      if (g->done) break;
      g->iter += 1;
      if (!isfinite(s[0])) {
        g->done = BREAKDOWN;
      } else {
        g->beta = s[0] / g->rr;
        g->rr = s[0];
        if (s[0] <= g->tol2)
          g->done = CONVERGED;
        else if (g->iter >= g->max_iter)
          g->done = MAXITER;
      }
      break;
    }
    default:
      break;
  }
}

// Sum v[0..NV) over the block into thread 0 (fixed order); needs all threads.
template <int NV>
__device__ __forceinline__ void block_sum(double v[NV], double (*sh)[4]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k)
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], off);
  __syncthreads();
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < NV; ++k) sh[warp][k] = v[k];
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double a = 0.0;
      for (int w = 0; w < nw; ++w) a += sh[w][k];
      v[k] = a;
    }
  }
}

// Block partial of one right-hand side -> its slot in ra.partials.
// Must be reached by every thread of the block.
template <int NV>
__device__ __forceinline__ void block_partial(const RedArgs& ra, int rhs, int sb, int nblk, double v[NV]) {
  __shared__ double sh[32][4];
  block_sum<NV>(v, sh);
  if (threadIdx.x == 0)
#pragma unroll
    for (int k = 0; k < NV; ++k) ra.partials[((long)rhs * nblk + sb) * 4 + k] = v[k];
}

// After this block's partials are written: take a ticket; the last block of
// the grid sums every right-hand side's partials in a fixed order and runs
// the finalizer.  Must be reached by every thread of every block.
template <int NV>
__device__ void grid_finish(const RedArgs& ra, int nblk, int nrhs) {
  __shared__ double sh[32][4];
  __shared__ int is_last;
  if (threadIdx.x == 0) {
    __threadfence();
    unsigned t = atomicAdd(ra.counter, 1u);
    is_last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  for (int r = 0; r < nrhs; ++r) {
    double a[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) a[k] = 0.0;
    for (int b = threadIdx.x; b < nblk; b += blockDim.x)
#pragma unroll
      for (int k = 0; k < NV; ++k) a[k] += __ldcg(ra.partials + ((long)r * nblk + b) * 4 + k);
    block_sum<NV>(a, sh);
    if (threadIdx.x == 0) {
      double s[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
      for (int k = 0; k < NV; ++k) s[k] = a[k];
      finalize(ra, r, s);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) *ra.counter = 0u;
}

// Block partial -> global partial; the last block reduces and finalizes.
// Must be reached by every thread of every block.
template <int NV>
__device__ void reduce_finalize(const RedArgs& ra, int rhs, int sb, int nblk, int nrhs, double v[NV]) {
  block_partial<NV>(ra, rhs, sb, nblk, v);
  grid_finish<NV>(ra, nblk, nrhs);
}

}  // namespace bridge
