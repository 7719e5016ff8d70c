// Instantiations and launchers of the Moebius domain-wall kernels (dwf.cuh)
// for FP64 and FP32.
#include "kernels.h"

namespace bridge {

// Raise the kernel's dynamic shared memory limit to what this launch needs
// (once per kernel, device and size; the static shared memory of the fused
// reductions counts against the same per-block maximum).  `limit` is the
// caller's per-instantiation record of the limits set per device.
template <class K>
static void allow_smem(K kernel, long need, long (&limit)[64]) {
  if (need <= 48 * 1024) return;
  int dev = 0;
  cudaGetDevice(&dev);
  long& cur = limit[dev & 63];
  if (need <= cur) return;
  if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)need) == cudaSuccess) cur = need;
}

template <int P, bool M1, int M2, int EPI, int MINB, int SPT>
static bool go_hop1(const DwfArgs& a, cudaStream_t st) {
  static long limit[64] = {};
  auto k = dwf_hop_kernel<P, M1, M2, EPI, MINB, SPT>;
  const long smem = dwf_hop_smem(P, a.Ls, a.ns, M1, M2 == DM2_DENSE, a.fact != 0);
  allow_smem(k, smem, limit);
  k<<<a.nsb * a.nrhs, dwf_threads(a.ns, a.Ls / SPT), smem, st>>>(a);
  return true;
}

// Variant v -> (register budget MINB, slices per thread): 0 (2, 1), 1 (3, 1),
// 2 (4, 1), 3 (1, 2), 4 (2, 2), 5 (3, 2) for FP32 (two slices per thread need
// an even Ls); FP64 has only v = 0.
template <int P, bool M1, int M2, int EPI>
static bool go_hop(const DwfArgs& a, cudaStream_t st, int v) {
  if constexpr (P == P_F64) {
    return go_hop1<P, M1, M2, EPI, 1, 1>(a, st);
  } else {
    if (dwf_variant_spt(v, a.Ls) == 2) {
      if (v == 3) return go_hop1<P, M1, M2, EPI, 1, 2>(a, st);
      if (v == 5) return go_hop1<P, M1, M2, EPI, 3, 2>(a, st);
      return go_hop1<P, M1, M2, EPI, 2, 2>(a, st);
    }
    if (v == 1) return go_hop1<P, M1, M2, EPI, 3, 1>(a, st);
    if (v == 2) return go_hop1<P, M1, M2, EPI, 4, 1>(a, st);
    return go_hop1<P, M1, M2, EPI, 2, 1>(a, st);
  }
}

template <int P>
static bool hop_for(bool m1, int m2, int epi, const DwfArgs& a, cudaStream_t st, int v) {
  if (m1) {
    if (m2 == DM2_NONE && epi == DE_NONE) return go_hop<P, true, DM2_NONE, DE_NONE>(a, st, v);
    if (m2 == DM2_PLAIN && epi == DE_NONE) return go_hop<P, true, DM2_PLAIN, DE_NONE>(a, st, v);
    if (m2 == DM2_PLAIN && epi == DE_NORM) return go_hop<P, true, DM2_PLAIN, DE_NORM>(a, st, v);
    if (m2 == DM2_PLAIN && epi == DE_CGUPD) return go_hop<P, true, DM2_PLAIN, DE_CGUPD>(a, st, v);
    if (m2 == DM2_DENSE && epi == DE_NONE) return go_hop<P, true, DM2_DENSE, DE_NONE>(a, st, v);
  } else {
    if (m2 == DM2_NONE && epi == DE_NONE) return go_hop<P, false, DM2_NONE, DE_NONE>(a, st, v);
    if (m2 == DM2_DENSE && epi == DE_NONE) return go_hop<P, false, DM2_DENSE, DE_NONE>(a, st, v);
    if (m2 == DM2_DENSE && epi == DE_NORM) return go_hop<P, false, DM2_DENSE, DE_NORM>(a, st, v);
  }
  return false;
}

bool launch_dwf_hop(int prec, bool m1, int m2, int epi, const DwfArgs& a, cudaStream_t st, int variant) {
  switch (prec) {
    case P_F64: return hop_for<P_F64>(m1, m2, epi, a, st, variant);
    case P_F32: return hop_for<P_F32>(m1, m2, epi, a, st, variant);
  }
  return false;
}

template <int P, int MODE, int MINB>
static bool go_mix1(const DwfMixArgs& a, cudaStream_t st) {
  static long limit[64] = {};
  auto k = dwf_mix_kernel<P, MODE, MINB>;
  const long smem = dwf_mix_smem(P, a.Ls, a.ns, a.fact != 0);
  allow_smem(k, smem, limit);
  k<<<a.nsb * a.nrhs, dwf_threads(a.ns, a.Ls), smem, st>>>(a);
  return true;
}

template <int P, int MODE>
static bool go_mix(const DwfMixArgs& a, cudaStream_t st, int v) {
  if constexpr (P == P_F64) {
    return go_mix1<P, MODE, 1>(a, st);
  } else {
    if (v == 1) return go_mix1<P, MODE, 3>(a, st);
    if (v == 2) return go_mix1<P, MODE, 4>(a, st);
    return go_mix1<P, MODE, 2>(a, st);
  }
}

bool launch_dwf_mix(int prec, int mode, const DwfMixArgs& a, cudaStream_t st, int variant) {
  if (prec == P_F64) return mode == DX_CGP ? go_mix<P_F64, DX_CGP>(a, st, 0) : go_mix<P_F64, DX_PLAIN>(a, st, 0);
  if (prec == P_F32)
    return mode == DX_CGP ? go_mix<P_F32, DX_CGP>(a, st, variant) : go_mix<P_F32, DX_PLAIN>(a, st, variant);
  return false;
}

}  // namespace bridge
