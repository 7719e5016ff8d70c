// Host side of the Moebius domain-wall operator: parameter sets, operator
// application on five-dimensional fields and the mixed-precision CG solve.
// A five-dimensional field is a Field whose nrhs counts slices: slice
// q = rhs * Ls + s holds fifth coordinate s of right-hand side rhs.
#pragma once

#include "host.h"

namespace bridge {

bool op_is_mobius(const bridge_op& op);
// EINVAL unless Ls, M5, b5, c5, mf are usable.
void check_mobius(const bridge_op& op);
// The s-matrices for op's parameters (cached on the lattice).
std::shared_ptr<DwfSet> dwf_set(bridge_lattice_s* L, const bridge_op& op);

// Operators on five-dimensional fields (nrhs = right-hand sides x Ls),
// asynchronous on st.
void dwf_apply_d(bridge_lattice_s* L, const bridge_op& op, const Field& out, const Field& in, cudaStream_t st);
void dwf_apply_deo(bridge_lattice_s* L, const bridge_op& op, int out_parity, const Field& out, const Field& in,
                   cudaStream_t st);
void dwf_apply_dhat(bridge_lattice_s* L, const bridge_op& op, const Field& out, const Field& in, bool dagger,
                    cudaStream_t st);

// Time the launch shapes (threads per block, register budget) of the FP32
// kernels a solve with nrhs right-hand sides launches and keep the fastest
// in the lattice's shape table (no-op for FP64, whose kernels have one shape).
void tune_dwf_kernels(bridge_lattice_s* L, const bridge_op& op, int prec, int nrhs);

// Solve D x = b for nrhs five-dimensional right-hand sides: canonical FP64
// fields on the device (x: initial guess in, solution out).  Blocking.
// Returns the overall status and fills info[nrhs].
int dwf_solve(bridge_lattice_s* L, const bridge_op& op, const bridge_solver& prm, const double* b_dev, double* x_dev,
              int nrhs, bridge_info* info);

}  // namespace bridge
