/*
 * libbridge -- GPU (sm_103a) even-odd Wilson/clover Dirac operator and
 * mixed-precision BiCGStab solver, the fermion-propagator path of
 * "Bridge++ 2.0: Benchmark results on supercomputer Fugaku" (Sec. 2, Eq. 1,
 * Sec. 3).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Lattice: extents dims = {Lx, Ly, Lz, Lt}, all even and >= 2; site index
 *   i = x + Lx*(y + Ly*(z + Lz*t)); parity (x+y+z+t) mod 2, even = 0.
 * Canonical spinor layout (FP64): [rhs][t][z][y][x][spin 4][colour 3][re,im],
 *   i.e. 24 doubles per site.  A half-lattice vector holds the V/2 sites of
 *   one parity in increasing lexicographic order (site i sits at i/2).
 * Canonical link layout (FP64): [mu][t][z][y][x][row 3][col 3][re,im],
 *   mu = x, y, z, t; U_mu(x) connects x to x + mu.
 * Gamma matrices: chiral basis gamma_k = [[0, -i s_k], [i s_k, 0]] (k = x, y,
 *   z), gamma_t = [[0, 1], [1, 0]], gamma_5 = diag(1, 1, -1, -1).  (The paper
 *   uses the QWS convention and converts at its call boundary; the basis is
 *   not printed there.)
 * Operator: D = T - kappa H with
 *   (H psi)(x) = sum_mu (1 - gamma_mu) U_mu(x) psi(x+mu)
 *              + (1 + gamma_mu) U_mu(x-mu)^dagger psi(x-mu),
 *   a boundary phase bc[mu] (+1 periodic, -1 antiperiodic) on every hop that
 *   wraps, and T = 1 (Wilson) or T = 1 - kappa c_sw sum_{mu<nu} sigma_{mu nu}
 *   F_{mu nu} (clover; F from the four-leaf clover, made traceless).
 * Even-odd form (Eq. 1): D_ee = T_e, D_oo = T_o, D_eo = -kappa H_eo,
 *   D_oe = -kappa H_oe, D^(eo) = 1 - D_ee^-1 D_eo D_oo^-1 D_oe.
 *
 * Memory: pointer arguments named *_dev are device pointers (cudaMalloc,
 * cudaMallocAsync or a framework allocator on the current device); all
 * others are host pointers.  The library copies every input it keeps; the
 * caller owns every buffer it passes.  Device buffers must be 16-byte
 * aligned.
 *
 * Errors: every function returns BRIDGE_OK (0) or a negative status and never
 * aborts; bridge_last_error() gives a one-line description of the most recent
 * failure on the calling thread.  A lattice handle may be used from one host
 * thread at a time (calls are serialised by an internal lock); the request
 * API (bridge_submit .. bridge_request_release) is thread-safe.
 *
 * There is no CPU fallback: without a CUDA device of compute capability 10.3
 * bridge_lattice_create returns BRIDGE_ECUDA.
 */
#ifndef BRIDGE_H
#define BRIDGE_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bridge_lattice_s* bridge_lattice;  /* opaque, library-owned */
typedef struct bridge_field_s* bridge_field;      /* opaque, library-owned */
typedef struct bridge_request_s* bridge_request_h; /* opaque, library-owned */

enum bridge_status {
  BRIDGE_OK = 0,
  BRIDGE_PENDING = 1,
  BRIDGE_EINVAL = -1,     /* bad argument (null pointer, odd extent, unknown enum) */
  BRIDGE_ENOMEM = -2,     /* device allocation failed or request exceeds the memory budget */
  BRIDGE_ENOCONV = -3,    /* solver hit its iteration limit above tolerance */
  BRIDGE_EBREAKDOWN = -4, /* BiCGStab breakdown that restarts could not cure */
  BRIDGE_ETIMEDOUT = -5,  /* bridge_wait ran out of time (request still running) */
  BRIDGE_ECUDA = -6,      /* CUDA error (text in bridge_last_error) */
  BRIDGE_ESTATE = -7      /* call out of order (e.g. operator before gauge upload) */
};

/* Storage precision of a field or of an operator application.  F64 computes
 * in FP64; F32 stores and computes in FP32; F16/BF16 store spinors as 16-bit
 * values times a per-site FP32 scale (max |component|), links and clover
 * blocks as plain 16-bit values, and compute in FP32. */
enum bridge_prec { BRIDGE_F64 = 0, BRIDGE_F32 = 1, BRIDGE_F16 = 2, BRIDGE_BF16 = 3 };

enum bridge_kind { BRIDGE_WILSON = 0, BRIDGE_CLOVER = 1, BRIDGE_MOBIUS = 2, BRIDGE_STAGGERED = 3 };

/* Site subset of a field: one parity (half lattice) or the full lattice. */
enum bridge_subset { BRIDGE_EVEN = 0, BRIDGE_ODD = 1, BRIDGE_FULL = 2 };

/* Operator selector for bridge_apply. */
enum bridge_apply_op {
  BRIDGE_APPLY_D = 0,    /* full D, FULL -> FULL */
  BRIDGE_APPLY_DEO = 1,  /* D_eo = -kappa H_eo, ODD -> EVEN */
  BRIDGE_APPLY_DOE = 2,  /* D_oe = -kappa H_oe, EVEN -> ODD */
  BRIDGE_APPLY_DHAT = 3  /* D^(eo) of Eq. 1, EVEN -> EVEN */
};

typedef struct {
  int kind;     /* bridge_kind */
  double kappa; /* hopping parameter (WILSON, CLOVER) */
  double csw;   /* clover coefficient (CLOVER only) */
  int bc[4];    /* boundary phase per direction, +1 or -1; {1,1,1,-1} usual */
  /* MOBIUS only (Sec. 2: Moebius domain-wall fermions, the fifth coordinate
   * an inner index of each site).  With W = D_W(-M5) = (4 - M5) - H/2 and
   * (P psi)_s = P_- psi_{s+1} + P_+ psi_{s-1} (P_+- = (1 +- gamma_5)/2,
   * psi_{Ls} -> -mf psi_0, psi_{-1} -> -mf psi_{Ls-1}):
   *   D psi = (b5 W + 1) psi + (c5 W - 1) P psi;
   * b5 = 1, c5 = 0 is the Shamir operator.  Even-odd blocks (Eq. 1) by the
   * parity of the four-dimensional site: D_ee = D_oo = A = (b5 (4-M5) + 1)
   * + (c5 (4-M5) - 1) P, D_eo = -(1/2) H_eo B, D_oe = -(1/2) H_oe B with
   * B = b5 + c5 P.  Every spinor argument then holds Ls slices per
   * right-hand side, canonical layout [rhs][s][t][z][y][x][spin][colour][re,im]
   * (half-lattice vectors [rhs][s][sites of one parity][spin][colour][re,im]):
   * nrhs counts five-dimensional fields, and every buffer size stated below
   * for an operator or solve call is multiplied by Ls.  Computed in FP64 or
   * FP32 (prec / inner_prec F16 and BF16 return EINVAL); the solver is CG on
   * the normal equations of D^(eo) (Sec. 3 / Fig. 7 of the paper use CG for
   * this operator) inside the same FP64 defect correction.  bridge_apply
   * takes fields of nrhs x Ls slices.  Not accepted by
   * bridge_mult_Dhat_noalloc, bridge_tune or bridge_submit. */
  int Ls;       /* fifth extent, 1 .. 32 */
  double M5;    /* domain-wall height */
  double b5, c5; /* Moebius coefficients */
  double mf;    /* quark mass */
  /* STAGGERED only (Sec. 2: the staggered action).  With eta_0 = 1,
   * eta_1 = (-1)^x, eta_2 = (-1)^(x+y), eta_3 = (-1)^(x+y+z):
   *   D chi(x) = mass chi(x) + (1/2) sum_mu eta_mu(x) [U_mu(x) chi(x+mu)
   *                                                   - U_mu(x-mu)^dag chi(x-mu)],
   * boundary phases bc as above.  Spinor arguments hold one colour vector
   * per site: canonical layout [rhs][t][z][y][x][colour 3][re,im] (6 doubles
   * per site instead of 24).  Even-odd blocks (Eq. 1): D_ee = D_oo = mass,
   * D^(eo) = 1 - D_eo D_oe / mass^2.  The solver is CG on the Hermitian
   * positive definite mass^2 - D_eo D_oe (the even block of the normal
   * equations) inside the FP64 defect correction; F64 or F32 only.  Not
   * accepted by bridge_apply, bridge_mult_Dhat_noalloc, bridge_tune or
   * bridge_submit. */
  double mass;
} bridge_op;

typedef struct {
  double tol;        /* stop when ||b - D x|| <= tol ||b|| (FP64 true residual) */
  int max_iter;      /* limit on inner BiCGStab iterations, summed over restarts */
  int inner_prec;    /* bridge_prec of the inner solver (mixed = 1) */
  double inner_tol;  /* inner relative tolerance; <= 0 picks 1e-5 (F32), 2e-3 (F16/BF16) */
  int mixed;         /* 1: FP64 defect correction around an inner_prec solver; 0: plain FP64 */
  int check_every;   /* iterations between host convergence polls (<= 0: 16) */
  int use_graph;     /* 1: replay iteration batches as CUDA graphs */
  int max_outer;     /* limit on defect-correction passes (<= 0: 50) */
  int method;        /* WILSON/CLOVER inner solver: BRIDGE_METHOD_AUTO (0) BiCGStab, switching to CG on the
                        normal equations of the Schur system for the remaining passes once a BiCGStab pass
                        stagnates (1000 iterations with |r^| > 1e-2 |b^| at its end); BRIDGE_METHOD_BICGSTAB (1)
                        BiCGStab only; BRIDGE_METHOD_CGNR (2) CG on D^dag D^ only.  Other kinds ignore it. */
} bridge_solver;
enum bridge_method { BRIDGE_METHOD_AUTO = 0, BRIDGE_METHOD_BICGSTAB = 1, BRIDGE_METHOD_CGNR = 2 };

typedef struct {
  int status;               /* BRIDGE_OK, BRIDGE_ENOCONV or BRIDGE_EBREAKDOWN */
  int outer_iters;          /* defect-correction passes (true-residual evaluations - 1) */
  int inner_iters;          /* BiCGStab iterations summed over passes */
  int restarts;             /* inner solves that ended in breakdown */
  double true_rel_residual; /* ||b - D x|| / ||b|| in FP64 on the GPU */
  double seconds;           /* wall time of the solve */
  int cgnr_passes;          /* WILSON/CLOVER: defect-correction passes whose inner solve was CG on the
                               normal equations (inner_iters then counts CG iterations for them) */
} bridge_info;

typedef struct {
  const char* name;  /* kernel class */
  long launches;
  double bytes;      /* algorithmic bytes (each input read once, output written once) */
  double flops;      /* stated flop count (hop 1320 + 24 per site, clover 504, ...) */
  double ms;         /* event-timed milliseconds (only while profiling) */
} bridge_kstat;

/* ---- lattice ------------------------------------------------------------ */

/* Create a lattice handle on the current CUDA device.  dims: 4 even extents
 * >= 2 with V/2 < 2^31.  Allocates the handle and a CUDA stream; no field
 * memory yet.  Errors: EINVAL (dims), ECUDA (no sm_103 device). */
int bridge_lattice_create(const int dims[4], bridge_lattice* out);
/* Free the handle and everything it owns; ESTATE while engine requests on
 * it are still running. */
int bridge_lattice_destroy(bridge_lattice lat);
/* The cudaStream_t (as void*) on which all work of this lattice is ordered. */
void* bridge_lattice_stream(bridge_lattice lat);
/* Block the host until all work queued on the lattice stream is done. */
int bridge_sync(bridge_lattice lat);

/* Upload a gauge field (Sec. 2: the operators act on a given SU(3) field).
 * U: canonical FP64 links, 4*V*18 doubles, host (or device for _dev).  The
 * links are copied and stored as FP64 18-real planes; FP32/F16/BF16 12-real
 * copies and, for CLOVER, the clover term T and T^-1 (built in FP64 on the
 * GPU for kappa*c_sw of op) are made on first use.  op may be NULL. */
int bridge_gauge_upload(bridge_lattice lat, const double* U, const bridge_op* op);
int bridge_gauge_upload_dev(bridge_lattice lat, const double* U_dev, const bridge_op* op);

/* ---- operators on canonical FP64 buffers ----------------------------------- */

/* out = D in on the full lattice (Sec. 2: Wilson/clover multiplication),
 * computed in precision prec; in/out hold nrhs canonical full spinors
 * (nrhs*V*24 doubles).  nrhs = 0 is a no-op.  Synchronous. */
int bridge_mult_D(bridge_lattice lat, const bridge_op* op, int prec, const double* in, double* out, int nrhs);
/* Half-lattice hopping block (Eq. 1): out_parity 0 gives D_eo in (in odd,
 * out even), 1 gives D_oe in; D_eo = -kappa H_eo.  in/out: nrhs canonical
 * half-lattice vectors (nrhs*V/2*24 doubles).  Synchronous. */
int bridge_mult_Deo(bridge_lattice lat, const bridge_op* op, int prec, int out_parity, const double* in, double* out,
                    int nrhs);
/* Schur operator D^(eo) = 1 - D_ee^-1 D_eo D_oo^-1 D_oe of Eq. 1 on even
 * half-lattice vectors.  Synchronous. */
int bridge_mult_Dhat(bridge_lattice lat, const bridge_op* op, int prec, const double* in, double* out, int nrhs);
/* Adjoint of the Schur operator, (D^(eo))^dagger = 1 - D_oe^dag D_oo^-dag
 * D_eo^dag D_ee^-dag, on even half-lattice vectors (the normal-equation
 * operator of the CG solve is D^(eo)^dagger D^(eo)).  MOBIUS only; EINVAL for
 * WILSON and CLOVER.  Synchronous. */
int bridge_mult_Dhat_dag(bridge_lattice lat, const bridge_op* op, int prec, const double* in, double* out, int nrhs);
/* Same four, with device buffers; work is queued on the lattice stream and
 * the call returns without waiting (use bridge_sync or the stream). */
int bridge_mult_D_dev(bridge_lattice lat, const bridge_op* op, int prec, const double* in_dev, double* out_dev, int nrhs);
int bridge_mult_Deo_dev(bridge_lattice lat, const bridge_op* op, int prec, int out_parity, const double* in_dev,
                        double* out_dev, int nrhs);
int bridge_mult_Dhat_dev(bridge_lattice lat, const bridge_op* op, int prec, const double* in_dev, double* out_dev,
                         int nrhs);
int bridge_mult_Dhat_dag_dev(bridge_lattice lat, const bridge_op* op, int prec, const double* in_dev,
                             double* out_dev, int nrhs);

/* ---- operator without device allocation ------------------------------------- */

/* Size of the fixed device scratch array used by bridge_mult_Dhat_noalloc:
 * 64 MiB, held on every GPU that loads the library until the process exits. */
#define BRIDGE_NOALLOC_SCRATCH_BYTES (64L << 20)

/* The Schur operator of bridge_mult_Dhat_dev, for callers that cannot call
 * cudaMalloc while they apply the operator (for example an application that
 * reserves all device memory for its own pool at start-up, or a
 * latency-critical loop where an allocation, which may synchronize the
 * device, is not allowed).  The paper has no counterpart.
 *
 * in_dev / out_dev: nrhs canonical FP64 even half-lattice vectors on the
 * device (nrhs*V/2*24 doubles each), owned by the caller.  Its scratch (the
 * input, the odd intermediate and the output in the GPU layout of precision
 * prec: 3 * nrhs blocks of the half-lattice field size) lives in one fixed
 * file-scope device array of BRIDGE_NOALLOC_SCRATCH_BYTES; larger requests
 * return BRIDGE_EINVAL.  The call allocates nothing: the links in prec and,
 * for CLOVER, T^-1 for this kappa*c_sw in prec must already exist (apply the
 * operator once with bridge_mult_Dhat or bridge_solve in that precision
 * first), else BRIDGE_ESTATE.  The first call on each device looks up the
 * array's device address (and may load the library's device code there), so
 * make that first call during set-up.  Work is queued on the lattice stream
 * and the call returns without waiting.  All calls share the one array: calls
 * whose work overlaps on the GPU (for example on two lattices, whose streams
 * run concurrently) race on it; calls on one lattice are ordered by its
 * stream.  No part of the scratch needs to start at zero. */
int bridge_mult_Dhat_noalloc(bridge_lattice lat, const bridge_op* op, int prec, const double* in_dev, double* out_dev,
                             int nrhs);

/* ---- domain decomposition with halo exchange ------------------------------------ */

/* The lattice cut into nparts slabs along t, each a sub-lattice with its own
 * links, clover term, fields and stream, joined by a halo exchange on every
 * application of the hopping term -- the decomposition the paper runs over
 * MPI processes (Sec. 2: sub-lattices per process, boundary data exchanged
 * with the neighbours by persistent communication while the bulk is
 * computed; Sec. 3: weak and strong scaling).  Per hop term: the interior
 * stencil of every slab (t hops leaving the slab left out) overlaps, on a
 * second stream per slab, the packing of the two faces -- (1 - gamma_t) psi
 * of the first time slice and U_t^dagger (1 + gamma_t) psi of the last, six
 * complex numbers per face site -- and their copy into the neighbours'
 * receive buffers; a boundary kernel then adds the crossing hops
 * (reconstructed to four spin components, times beta, the global boundary
 * phase where the hop wraps, and T^-1 for a T^-1 epilogue).  Dot products
 * are per-slab partial sums added over all slabs.  Here the slabs share the
 * caller's GPU and the exchange is a device-to-device copy. */
typedef struct bridge_dd_s* bridge_dd;

/* The face schedule of one slab (host arithmetic only, no device needed). */
typedef struct {
  int local_dims[4];       /* Lx, Ly, Lz, Lt / nparts */
  int t0;                  /* first global time slice of the slab */
  int rank_up;             /* slab holding time slice t0 + Lt / nparts (mod Lt): receives this slab's
                              last-slice face, sends its first-slice face here */
  int rank_down;           /* slab holding time slice t0 - 1 (mod Lt) */
  long face_sites;         /* sites per parity of one time slice, Lx Ly Lz / 2; face site f of a slice is
                              the site of that parity whose spatial lexicographic index s has s / 2 = f */
  int up_wraps;            /* 1: forward t hops out of this slab cross the lattice boundary (phase bc[3]) */
  int down_wraps;          /* 1: backward t hops out of this slab cross the lattice boundary */
  long canon_offset_sites; /* lexicographic index of the slab's first site in the global lattice */
} bridge_dd_plan;

/* Face schedule of slab `rank` for global extents dims cut into nparts slabs.
 * EINVAL unless every extent is even and >= 2 and Lt / nparts is even. */
int bridge_dd_plan_of(const int dims[4], int nparts, int rank, bridge_dd_plan* plan);
/* Decompose lattice lat (gauge field uploaded) for operator op (WILSON or
 * CLOVER; the clover term is taken from the whole field) into nparts slabs.
 * The handle refers to lat, which must outlive it.  Synchronous.  Errors:
 * EINVAL (kind, bc, nparts), ESTATE (no gauge field), ENOMEM. */
int bridge_dd_create(bridge_lattice lat, const bridge_op* op, int nparts, bridge_dd* out);
int bridge_dd_destroy(bridge_dd dd);
/* The operators of bridge_mult_D_dev / _Deo_dev / _Dhat_dev (same canonical
 * device layouts, nrhs right-hand sides, any precision) through the
 * decomposition.  Synchronous. */
int bridge_dd_mult_D_dev(bridge_dd dd, int prec, const double* in_dev, double* out_dev, int nrhs);
int bridge_dd_mult_Deo_dev(bridge_dd dd, int prec, int out_parity, const double* in_dev, double* out_dev, int nrhs);
int bridge_dd_mult_Dhat_dev(bridge_dd dd, int prec, const double* in_dev, double* out_dev, int nrhs);
/* Plain FP64 BiCGStab on the even-odd system of Eq. 1 over the slabs (every
 * dot product summed over all slabs), solved to 0.1 s->tol in the Schur
 * residual, then x_o reconstructed and the FP64 true residual ||b - D x|| /
 * ||b|| of the whole lattice reported in info (status OK when it is <=
 * s->tol).  b_dev / x_dev: canonical full fields on the device; x starts
 * from zero.  Uses s->tol and s->max_iter only.  Synchronous. */
int bridge_dd_solve_dev(bridge_dd dd, const bridge_solver* s, const double* b_dev, double* x_dev, int nrhs,
                        bridge_info* info);

/* ---- solver ------------------------------------------------------------------ */

/* Solve D x = b for nrhs right-hand sides (Sec. 3: BiCGStab for the clover
 * operator; mixed-precision BiCGStab for propagators).  Even-odd
 * preconditioned BiCGStab on D^(eo) (Eq. 1) inside an FP64 defect-correction
 * loop on the true residual.  b, x: canonical full spinors, nrhs*V*24
 * doubles each; x holds the initial guess on entry (zeros for none) and the
 * solution on return.  info: array of nrhs records (may be NULL).
 * Returns OK when every right-hand side reached tol, else ENOCONV or
 * EBREAKDOWN (x then holds the best iterate).  Synchronous. */
int bridge_solve(bridge_lattice lat, const bridge_op* op, const bridge_solver* s, const double* b, double* x, int nrhs,
                 bridge_info* info);
int bridge_solve_dev(bridge_lattice lat, const bridge_op* op, const bridge_solver* s, const double* b_dev,
                     double* x_dev, int nrhs, bridge_info* info);
/* Defaults: tol 1e-10, max_iter 20000, F32 inner, mixed, poll every 16, graphs on. */
void bridge_solver_defaults(bridge_solver* s);

/* Autotune (the GPU counterpart of the paper's site-tile study, Sec. 3 /
 * Fig. 5): time the hop and vector kernels a solve with this operator,
 * inner precision prec and nrhs right-hand sides will launch, over block
 * sizes and grid shapes, on scratch buffers, and keep the fastest shape per
 * kernel for this lattice.  With the environment variable BRIDGE_TUNE_CACHE
 * naming a file, results are appended there and loaded by later
 * bridge_lattice_create calls on the same device model.  Synchronous. */
int bridge_tune(bridge_lattice lat, const bridge_op* op, int prec, int nrhs);
/* The current shape table as text ("key block nblk variant" per line) in
 * out[n]; returns the full length. */
int bridge_tune_table(bridge_lattice lat, char* out, int n);
/* Set one entry of the shape table (key as printed by bridge_tune_table):
 * block in [64, 256] (multiple of 32), nblk >= 1 site blocks per
 * right-hand-side group, variant in [0, 12] (register budget / read-once
 * loads for 0-5, 2-4 right-hand sides per thread for 6-8, the shared-link
 * tile kernel for 9-10, the same with pipelined neighbour loads for 11-12,
 * FP16/BF16 storage only; a variant a kernel does not have falls back to
 * 0).  Lets tests and users pin a launch shape; EINVAL for values out of
 * range. */
int bridge_tune_set(bridge_lattice lat, const char* key, int block, int nblk, int variant);

/* ---- fields in the GPU layout (resident data) ------------------------------- */

/* A library-owned device field of nrhs spinors in the GPU site layout of
 * precision prec over subset (bridge_subset). */
int bridge_field_create(bridge_lattice lat, int prec, int subset, int nrhs, bridge_field* out);
int bridge_field_destroy(bridge_field f);
/* Fill from / copy to canonical FP64 (full or half-lattice per the field's
 * subset); src/dst on the device if on_device != 0, else on the host.
 * Device-side copies are queued on the lattice stream; host-side ones block. */
int bridge_field_import(bridge_field f, const double* src, int on_device);
int bridge_field_export(bridge_field f, double* dst, int on_device);
/* out = op(in) in the fields' precision (both fields must share it); queued
 * on the lattice stream.  See bridge_apply_op for the subsets required. */
int bridge_apply(bridge_lattice lat, const bridge_op* op, int which, bridge_field out, bridge_field in);

/* ---- two-level multigrid ------------------------------------------------------- */

/* The multigrid solver of Sec. 3 (a two-level DD-alpha-AMG variant): an outer
 * Flexible BiCGStab in FP64 on D, preconditioned by an FP32 cycle made of a
 * coarse-grid correction (BiCGStab on the coarse operator to coarse_tol) and
 * SAP post-smoothing (sap_cycles cycles; blocks coloured by the parity of
 * their block coordinates; each block system solved by mr_steps
 * minimal-residual steps on D restricted to the block).  Aggregates are one
 * block and one chirality; the prolongation's columns are the null vectors
 * orthonormalised per aggregate (Gram-Schmidt in the given order); the
 * coarse operator is P^dag D P (nine couplings per coarse site: the block
 * and its eight neighbours).  WILSON and CLOVER operators. */
typedef struct bridge_mg_s* bridge_mg; /* opaque, library-owned */

typedef struct {
  int block[4];       /* block extents; each divides the lattice with an even quotient; 2 .. 256 sites */
  int nvec;           /* null vectors, 1 .. 32 */
  double setup_tol;   /* tolerance of the generated null vectors' solves D v = eta (random eta) */
  int setup_steps;    /* inverse-iteration steps per generated null vector (v <- D^-1 v / |v|) */
  int sap_cycles;     /* SAP post-smoothing cycles per preconditioner application */
  int mr_steps;       /* minimal-residual steps per block system */
  double coarse_tol;  /* relative tolerance of the coarse BiCGStab */
  int coarse_maxiter; /* iteration limit of the coarse BiCGStab */
  int coarse_half;    /* 1: the coarse BiCGStab reads an FP16 copy of the coarse operator (FP32 math) */
  int coarse_eo;      /* 1: with coarse_half and 2 nvec in {8, 16, 24, 32, 48}, the coarse BiCGStab runs on
                         the even-odd preconditioned coarse system (coarse sites split by the parity of
                         their block coordinates; every hopping coupling joins the two), the odd part
                         reconstructed after; coarse_tol then bounds that system's relative residual */
} bridge_mg_params;

/* Defaults: blocks 4^4, 16 null vectors, setup_tol 5e-2, 1 setup step,
 * 2 SAP cycles, 4 MR steps, coarse_tol 5e-2, coarse_maxiter 200, FP16
 * coarse operator in the coarse solver, even-odd coarse system. */
void bridge_mg_defaults(bridge_mg_params* p);
/* Build the multigrid hierarchy for op on the lattice's gauge field.
 * null_vectors: NULL to generate them (solves of random sources), or nvec
 * canonical full spinors on the host (nvec*V*24 doubles), used as given.
 * The handle keeps pointers to the lattice, which must outlive it.
 * Synchronous.  Errors: EINVAL (blocks, counts, operator kind), ESTATE (no gauge). */
int bridge_mg_setup(bridge_lattice lat, const bridge_op* op, const bridge_mg_params* p, const double* null_vectors,
                    bridge_mg* out);
int bridge_mg_destroy(bridge_mg mg);
/* Solve D x = b for nrhs right-hand sides (host canonical buffers; x holds
 * the initial guesses) to s->tol in the true FP64 residual: FP64 defect
 * correction (at most s->max_outer passes) around FP32 FBiCGStab passes
 * preconditioned by the cycle (at most s->max_iter FBiCGStab iterations in
 * all; a pass stops at s->inner_tol, default 1e-6, or at the reduction the
 * true residual still needs).  info[nrhs]: status, passes in outer_iters,
 * FBiCGStab iterations in inner_iters, restarts, true residual, seconds.
 * Synchronous. */
int bridge_mg_solve(bridge_mg mg, const bridge_solver* s, const double* b, double* x, int nrhs, bridge_info* info);
/* The same on device buffers (queued on the lattice stream; returns when done). */
int bridge_mg_solve_dev(bridge_mg mg, const bridge_solver* s, const double* b_dev, double* x_dev, int nrhs,
                        bridge_info* info);

/* Pieces of the cycle, on host canonical buffers, for tests.  Coarse
 * vectors are [block][chirality][vector] complex ([re, im] doubles), blocks
 * ordered x fastest. */
enum bridge_mg_apply_op {
  BRIDGE_MG_RESTRICT = 0, /* fine in -> coarse out: P^dag in */
  BRIDGE_MG_PROLONG = 1,  /* coarse in -> fine out: P in */
  BRIDGE_MG_COARSE = 2,   /* coarse -> coarse: D_c in (the FP32 coarse operator) */
  BRIDGE_MG_SAP = 3,      /* fine -> fine: sap_cycles SAP cycles on D x = in from x = 0 */
  BRIDGE_MG_CYCLE = 4,    /* fine -> fine: the preconditioner */
  BRIDGE_MG_COARSE_HALF = 5, /* coarse -> coarse: D_c in with the FP16 copy the coarse solver uses
                                (EINVAL when the setup ran with coarse_half = 0) */
  BRIDGE_MG_COARSE_SOLVE = 6 /* coarse -> coarse: the coarse solver's approximation of D_c^-1 in */
};
int bridge_mg_apply(bridge_mg mg, int which, const double* in, double* out);
/* The coarse operator: [block][coupling 9][column][row] complex doubles;
 * coupling 0 is the block itself, 1 + 2 mu / 2 + 2 mu the blocks at +mu / -mu. */
int bridge_mg_coarse_matrix(bridge_mg mg, double* out);
int bridge_mg_info(bridge_mg mg, int* nblocks, int* nvec);
/* Coarse solves run so far and their BiCGStab iterations in total. */
int bridge_mg_counters(bridge_mg mg, long* coarse_solves, long* coarse_iters);

/* ---- serving: continuous batching of solve requests ------------------------- */

/* Limits of the request engine: total device bytes that admitted requests
 * may hold (0 = 80% of free memory at first use) and the maximum number of
 * requests on the GPU at once (<= 0: 64).  Call before the first submit. */
int bridge_engine_config(size_t memory_budget_bytes, int max_active);
/* Queue a solve of D x = b (as bridge_solve, x0 = 0).  b is copied; the
 * request is admitted when memory and a slot are free (requests that fit may
 * pass older ones that do not, until the oldest has waited 2 s) and then
 * advances concurrently with the other admitted requests, each on its own
 * stream; smaller requests get higher stream priority.
 * The lattice must outlive the request.  Errors: EINVAL, ENOMEM (request
 * larger than the whole budget). */
int bridge_submit(bridge_lattice lat, const bridge_op* op, const bridge_solver* s, const double* b, int nrhs,
                  bridge_request_h* out);
/* As bridge_submit, but b is borrowed, not copied: the caller keeps it valid
 * and unchanged until the request has finished (bridge_poll / bridge_wait
 * returned its final status) or has been released (bridge_request_release
 * returns only once a borrowed b is no longer read).  A queue of waiting
 * requests then holds no host copies of its right-hand sides. */
int bridge_submit_borrowed(bridge_lattice lat, const bridge_op* op, const bridge_solver* s, const double* b,
                           int nrhs, bridge_request_h* out);
/* PENDING while running; else the request's final status, with x_out
 * (nrhs*V*24 doubles, may be NULL) and info[nrhs] (may be NULL) filled. */
int bridge_poll(bridge_request_h h, double* x_out, bridge_info* info);
/* As bridge_poll, blocking up to timeout_ms (< 0: forever); ETIMEDOUT if
 * the request is still running. */
int bridge_wait(bridge_request_h h, int timeout_ms, double* x_out, bridge_info* info);
/* Free a finished request; a running one is cancelled first. */
int bridge_request_release(bridge_request_h h);
/* Timestamps (seconds, monotonic clock) of submit, admission and completion. */
int bridge_request_times(bridge_request_h h, double* t_submit, double* t_admit, double* t_done);

/* ---- diagnostics --------------------------------------------------------- */

const char* bridge_strerror(int status);
const char* bridge_last_error(void);
/* Kernel statistics of this lattice since the last reset: out[k] for the
 * first min(n, count) classes; returns the number of classes. */
int bridge_stats(bridge_lattice lat, bridge_kstat* out, int n);
int bridge_stats_reset(bridge_lattice lat);
/* While enabled, every kernel launch of this lattice is bracketed by CUDA
 * events on its stream and graphs are not used; bridge_stats then reports
 * event-timed milliseconds per class. */
int bridge_profile(bridge_lattice lat, int enable);
/* Number of kernels this library launched in this process (graph nodes
 * count once per replay). */
long bridge_launch_count(void);
/* Number of device allocations (cudaMalloc and stream-ordered cudaMallocAsync)
 * this library made in this process; a diagnostic for tests of the
 * no-allocation entry point. */
long bridge_device_alloc_count(void);
/* Measured arithmetic throughput of the current device's scalar fused
 * multiply-add pipe (the instruction the stencils use), for the rooflines
 * of kernels bound by arithmetic rather than memory; the paper has no
 * counterpart (it quotes A64FX's nominal peak).  prec: BRIDGE_F32 or
 * BRIDGE_F64.  *flops_per_s = 2 x FMAs per second of a grid that fills every
 * SM with independent FMA chains, best of five timed launches.  Runs a few
 * milliseconds of GPU work on a private stream and synchronizes it.
 * Returns BRIDGE_EINVAL for another precision or a NULL pointer,
 * BRIDGE_ECUDA without a device. */
int bridge_alu_peak(int prec, double* flops_per_s);
/* Neighbour map of the GPU layout, computed on the host with the same code
 * the kernels use: out[2*mu + 0/1] = half-lattice index of x + mu / x - mu
 * for half-lattice site ih of the given parity; wraps[mu*2 + 0/1] = 1 when
 * that hop crosses the boundary.  For tests of the index arithmetic. */
int bridge_debug_neighbours(const int dims[4], int parity, long ih, long out[8], int wraps[8]);

#ifdef __cplusplus
}
#endif

#endif /* BRIDGE_H */
