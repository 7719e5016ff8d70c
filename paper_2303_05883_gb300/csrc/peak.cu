// Arithmetic throughput of this GPU's FP32 and FP64 FMA pipes, measured the
// way the stencil kernels use them (scalar fused multiply-adds), for the
// rooflines of the kernels that are bound by arithmetic rather than by HBM.
//
// Every thread runs eight independent FMA chains (enough instruction-level
// parallelism to cover the pipe latency) over a fixed number of steps; the
// grid fills every SM with resident 256-thread blocks.  The result of each
// thread is stored so that the chains cannot be removed, and the store is a
// negligible fraction of the run time.  flops = 2 x FMAs; best of five timed
// launches after one warm-up.
#include <algorithm>

#include "host.h"

namespace bridge {

template <class R, int STEPS>
__global__ void __launch_bounds__(256) k_fma_chains(R* out, R m, R c) {
  R a[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) a[k] = (R)(threadIdx.x + k);
#pragma unroll 4
  for (int i = 0; i < STEPS; ++i)
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = fmar<R>(a[k], m, c);
  R s = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += a[k];
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <class R, int STEPS>
static double measure(cudaStream_t st) {
  int per_sm = 0;
  BR_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fma_chains<R, STEPS>, 256, 0));
  const int blocks = sm_count() * std::max(1, per_sm);
  DevBuf out((size_t)blocks * 256 * sizeof(R));
  cudaEvent_t e0, e1;
  BR_CUDA(cudaEventCreate(&e0));
  BR_CUDA(cudaEventCreate(&e1));
  float best = 1e30f;
  for (int rep = 0; rep < 6; ++rep) {
    BR_CUDA(cudaEventRecord(e0, st));
    k_fma_chains<R, STEPS><<<blocks, 256, 0, st>>>(reinterpret_cast<R*>(out.ptr), (R)0.9999, (R)1e-4);
    BR_CUDA(cudaEventRecord(e1, st));
    BR_CUDA(cudaEventSynchronize(e1));
    float ms = 0;
    BR_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    if (rep > 0) best = std::min(best, ms);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  BR_CUDA(cudaGetLastError());
  const double flops = 2.0 * 8.0 * STEPS * (double)blocks * 256;
  return flops / (best * 1e-3);
}

}  // namespace bridge

using namespace bridge;

extern "C" int bridge_alu_peak(int prec, double* flops_per_s) {
  try {
    if (!flops_per_s || (prec != BRIDGE_F64 && prec != BRIDGE_F32)) return BRIDGE_EINVAL;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
      cudaGetLastError();
      set_error(BRIDGE_ECUDA, "no CUDA device");
      return BRIDGE_ECUDA;
    }
    cudaStream_t st;
    BR_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    double v = 0;
    try {
      v = prec == BRIDGE_F32 ? measure<float, 8192>(st) : measure<double, 256>(st);
    } catch (...) {
      cudaStreamDestroy(st);
      throw;
    }
    cudaStreamDestroy(st);
    *flops_per_s = v;
  } catch (const Error& e) {
    set_error(e.code, e.msg);
    return e.code;
  }
  return BRIDGE_OK;
}
