// Host-visible declarations of the kernel launchers (implemented in the .cu
// translation units) used by the lattice, operator and solver code.
#pragma once

#include "dslash.cuh"
#include "dwf.cuh"

namespace bridge {

// ---------------------------------------------------------------- hop
bool launch_hop_any(int prec, int flags, int red, const HopArgs& a, int block, cudaStream_t st, int* occ = nullptr,
                    int variant = 0);

// ------------------------------------------------ Moebius domain wall
// Combinations instantiated (m1, m2, epi): (1, NONE, NONE), (1, PLAIN, NONE),
// (1, PLAIN, NORM), (1, PLAIN, CGUPD), (1, DENSE, NONE), (0, NONE, NONE),
// (0, DENSE, NONE), (0, DENSE, NORM); F64 and F32.  false for any other.
// variant: register budget of the FP32 kernels, 0/1/2 = at most 128/85/64
// registers per thread, 3/4/5 = two slices per thread with no cap / <= 128 /
// <= 85 registers (FP64: one variant).
// Variants 3-5: two fifth-dimension slices per thread (even Ls; an odd Ls
// runs them as one slice per thread).
constexpr int DWF_NVARIANT = 6;
inline int dwf_variant_spt(int variant, int Ls) { return (variant >= 3 && Ls % 2 == 0) ? 2 : 1; }
bool launch_dwf_hop(int prec, bool m1, int m2, int epi, const DwfArgs& a, cudaStream_t st, int variant = 0);
bool launch_dwf_mix(int prec, int mode, const DwfMixArgs& a, cudaStream_t st, int variant = 0);

// ----------------------------------------------------- BiCGStab vectors
enum BlasOp { B_INIT = 0, B_S = 1, B_XR = 2, B_P = 3, B_CG_INIT = 4, B_CG_XR = 5, B_CG_P = 6 };
struct BlasArgs {
  uint32_t vh;
  int nrhs, nblk;
  char* x;  // precision px
  long x_rs;
  char *r, *p, *v, *s, *t, *rhat;
  long r_rs, p_rs, v_rs, s_rs, t_rs, rhat_rs;
  const char* b;
  long b_rs;
  RedArgs red;
};
// B_INIT: x = 0, r = rhat = p = b, |b|^2 -> FIN_INIT
// B_S:    s = r - alpha v
// B_XR:   x += alpha p + omega s, r = s - omega t, (<rhat, r>, |r|^2) -> FIN_RHO
// B_P:    p = r + beta (p - omega v)
// B_CG_INIT, B_CG_XR, B_CG_P: CG on the normal equations of the Schur system
// (x = 0, p = r, |r|^2; x += alpha p, r -= alpha t, |r|^2; p = r + beta p),
// scalars in red.cg
bool launch_blas(int op, int prec, int px, const BlasArgs& a, int block, cudaStream_t st, int* occ = nullptr);

// ------------------------------------------------------------ layout
struct CopyArgs {
  uint32_t vh;
  int nrhs, nblk;
  int parity;   // parity of the half-lattice block (full-canonical conversions)
  Geom g;
  long V;       // full volume (canonical full-lattice strides)
  const double* canon;  // canonical FP64 (re, im) pairs
  double* canon_out;
  int canon_full;       // 1: canonical is a full-lattice field, 0: a half-lattice one
  long canon_rs;        // double2 entries between right-hand sides of canon / canon_out (0: 12 x sites)
  const char* src;
  long src_rs;
  char* dst;
  long dst_rs;
  const int* mask;      // per rhs; 0 -> write zeros (may be null)
  RedArgs red;          // norm of the source (FIN_STORE) when red.partials != null
};
bool launch_canon_to_field(int prec, const CopyArgs& a, int block, cudaStream_t st);
bool launch_field_to_canon(int prec, const CopyArgs& a, int block, cudaStream_t st);
bool launch_convert(int ps, int pd, const CopyArgs& a, int block, cudaStream_t st);   // dst = mask ? src : 0
bool launch_accumulate64(int ps, const CopyArgs& a, int block, cudaStream_t st);      // dst(F64) += src
bool launch_norm2(int prec, const CopyArgs& a, int block, cudaStream_t st);           // |src|^2 -> FIN_STORE
bool launch_clover_site(int prec, const CopyArgs& a, const char* clov, int block, cudaStream_t st);  // dst = A src
// dst = gamma5 A src (clov = null: gamma5 src); skips right-hand sides whose
// CG solve ended (red.cg with check_done)
bool launch_g5_site(int prec, const CopyArgs& a, const char* clov, int block, cudaStream_t st);

// ------------------------------------------------------- gauge, clover
// Canonical FP64 links (4, V, 3, 3) -> internal F64 blocks [parity][mu].
void launch_gauge_from_canon(const double* U, const Geom& g, char* g64, cudaStream_t st);
// Internal F64 links -> internal links of another precision.
bool launch_gauge_convert(int prec, const Geom& g, const char* g64, char* gp, cudaStream_t st);
// Clover term T = 1 - kcsw * sum sigma F and its inverse, packed FP64 [parity].
void launch_clover_build(const Geom& g, const char* g64, double kcsw, char* T64, char* Tinv64, cudaStream_t st);
bool launch_clover_convert(int prec, const Geom& g, const char* c64, char* cp, cudaStream_t st);

}  // namespace bridge
