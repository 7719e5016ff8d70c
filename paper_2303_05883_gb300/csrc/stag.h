// Host side of the staggered operator: fields, operator application and the
// mixed-precision CG solve.  A staggered field is a Field whose blocks hold
// one colour vector per site (stag.cuh layout); nrhs counts right-hand sides.
#pragma once

#include "host.h"

namespace bridge {

bool op_is_staggered(const bridge_op& op);
// EINVAL unless op.mass is finite and nonzero.
void check_staggered(const bridge_op& op);
Field make_stag_field(int prec, int subset, int nrhs, long vh);
Field& stag_workspace(bridge_lattice_s* L, const std::string& name, int prec, int subset, int nrhs);

// Canonical FP64 colour vectors on the device ([rhs][site][colour][re, im];
// full lattice or the sites of one parity) <-> a field.
void stag_canon_to_field(bridge_lattice_s* L, const double* canon, const Field& f, bool canon_full, cudaStream_t st);
void stag_field_to_canon(bridge_lattice_s* L, const Field& f, double* canon, bool canon_full, cudaStream_t st);

// D, D_eo / D_oe and the Schur operator of Eq. 1, asynchronous on st.
void stag_apply_d(bridge_lattice_s* L, const bridge_op& op, const Field& out, const Field& in, cudaStream_t st);
void stag_apply_deo(bridge_lattice_s* L, const bridge_op& op, int out_parity, const Field& out, const Field& in,
                    cudaStream_t st);
void stag_apply_dhat(bridge_lattice_s* L, const bridge_op& op, const Field& out, const Field& in, cudaStream_t st);

// Solve D x = b (canonical FP64 device buffers, x: guess in, solution out).
int stag_solve(bridge_lattice_s* L, const bridge_op& op, const bridge_solver& prm, const double* b_dev, double* x_dev,
               int nrhs, bridge_info* info);

}  // namespace bridge
