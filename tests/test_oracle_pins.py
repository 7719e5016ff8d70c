"""The FP64 oracle against closed forms, invariants and library routines.

No GPU: these pin the oracle to the mathematics of the Wilson/clover
operator (Sec. 2), the even-odd decomposition (Eq. 1) and the solve of
D x = b (Sec. 3) before any CUDA result is compared with it.
"""

import numpy as np
import pytest

import synth
from oracle import dirac, evenodd, solvers
from oracle.lattice import Lattice
from tests import pins


def test_gamma_basis_clifford_hermitian_gamma5():
    assert pins.gamma_algebra_error() < 1e-15


def test_sigma_block_diagonal_and_hermitian():
    from oracle import gamma

    for mu in range(4):
        for nu in range(mu + 1, 4):
            s = gamma.sigma(mu, nu)
            assert np.abs(s - s.conj().T).max() < 1e-15
            assert np.abs(s[:2, 2:]).max() == 0 and np.abs(s[2:, :2]).max() == 0


def test_free_field_plane_wave_closed_form():
    assert pins.free_field_error() < 1e-13


def test_free_field_inverse_closed_form():
    assert pins.free_field_inverse_error() < 1e-11


def test_gamma5_hermiticity_wilson_and_clover():
    assert pins.gamma5_hermiticity_error() < 1e-14
    assert pins.gamma5_hermiticity_error(csw=0.0) < 1e-14


def test_gauge_covariance():
    assert pins.covariance_error() < 1e-13


def test_plaquette_gauge_invariant_and_unit_for_free_field():
    dims = (4, 4, 2, 4)
    lat = Lattice(dims)
    U = synth.gauge_field(dims, 0.4, 3)
    Om = pins.random_su3(lat.V, np.random.default_rng(1))
    Ug = pins.gauge_transform(U, lat, Om)
    assert abs(dirac.plaquette(U, lat) - dirac.plaquette(Ug, lat)) < 1e-14
    assert abs(dirac.plaquette(synth.unit_gauge(dims), lat) - 1.0) < 1e-15


def test_abelian_flux_field_strength_and_clover_term():
    assert pins.abelian_flux_error() < 1e-13


def test_clover_term_trivial_cases_and_structure():
    dims = (4, 4, 4, 2)
    lat = Lattice(dims)
    U = synth.gauge_field(dims, 0.5, 9)
    T0 = dirac.clover_term(U, lat, 0.12, 0.0)
    assert np.abs(T0 - np.eye(12)).max() == 0
    T1 = dirac.clover_term(synth.unit_gauge(dims), lat, 0.12, 1.0)
    assert np.abs(T1 - np.eye(12)).max() < 1e-15
    T = dirac.clover_term(U, lat, 0.12, 1.0)
    assert np.abs(T - np.conj(np.swapaxes(T, 1, 2))).max() < 1e-15  # Hermitian
    g5 = np.kron(np.diag([1, 1, -1, -1]), np.eye(3))
    assert np.abs(T @ g5 - g5 @ T).max() < 1e-15  # commutes with gamma_5: 2 blocks of 6x6
    assert np.abs(T - np.eye(12)).max() > 1e-3


def test_blocks_reassemble_full_operator():
    assert pins.blocks_vs_full_error() < 1e-14


def test_dense_matrix_elements_equal_stencil():
    assert pins.dense_vs_stencil_error() < 1e-15


def test_schur_complement_dense_2x2x2x2():
    assert pins.schur_dense_error() < 1e-13


@pytest.mark.slow
def test_schur_complement_dense_4x2x2x2():
    assert pins.schur_dense_error(dims=(4, 2, 2, 2), seed=32) < 1e-13


def test_bicgstab_matches_dense_lu_full():
    assert pins.lu_vs_bicgstab_error() < 1e-12


def test_bicgstab_matches_dense_lu_evenodd():
    assert pins.lu_vs_bicgstab_error(evenodd_solve=True) < 1e-12


def test_evenodd_solve_equals_full_solve():
    assert pins.evenodd_vs_full_error() < 1e-10


def test_bicgstab_zero_source_and_restart_path():
    dims = (2, 2, 2, 2)
    lat = Lattice(dims)
    U = synth.gauge_field(dims, 0.3, 2)
    A = lambda v: dirac.dirac(U, v, lat, 0.12, 1.0)  # noqa: E731
    x, info = solvers.bicgstab(A, np.zeros((lat.V, 4, 3), dtype=np.complex128))
    assert info["converged"] and np.abs(x).max() == 0
    b = synth.gaussian_spinor(dims, 4)
    x, info = solvers.bicgstab(A, b, tol=1e-12, maxiter=3)
    assert not info["converged"] and info["iters"] == 3


def test_gauge_generator_su3():
    dims = (4, 2, 2, 2)
    U = synth.gauge_field(dims, 0.3, 5).reshape(-1, 3, 3)
    eye = np.eye(3)
    assert np.abs(np.conj(np.swapaxes(U, 1, 2)) @ U - eye).max() < 1e-14
    assert np.abs(np.linalg.det(U) - 1).max() < 1e-14
    U0 = synth.gauge_field(dims, 1e-9, 5).reshape(-1, 3, 3)
    assert np.abs(U0 - eye).max() < 1e-8
    # exp(i eps A) agrees with the eigen-decomposition form V diag(e^{i eps l}) V^dagger
    gen = synth.rng(5, synth.FIELD_GAUGE)
    A = synth.lie_gaussian(gen, 16)
    w, Vv = np.linalg.eigh(A)
    E = Vv @ (np.exp(0.3j * w)[..., None] * np.conj(np.swapaxes(Vv, 1, 2)))
    assert np.abs(E - synth.reunitarize(synth.expi_hermitian(A, 0.3))).max() < 1e-14


def test_lattice_rejects_odd_extent():
    with pytest.raises(ValueError):
        Lattice((4, 3, 4, 4))


def test_half_lattice_order_matches_lexicographic():
    lat = Lattice((4, 6, 2, 4))
    for p in (0, 1):
        s = lat.sites_of(p)
        assert np.all(np.diff(s) > 0) and len(s) == lat.V // 2
        # the k-th site of one parity is lexicographic index 2k or 2k+1
        assert np.all(s // 2 == np.arange(lat.V // 2))


# --- Moebius domain wall and CG (Sec. 2 operators, Sec. 3 / Fig. 7 solver) -----------


def test_mobius_overlap_relation_random_gauge():
    assert pins.mobius_overlap_error() < 1e-12


def test_mobius_free_field_overlap_closed_form():
    assert pins.mobius_free_field_error() < 1e-12


def test_mobius_schur_and_evenodd_solve_vs_dense():
    assert pins.mobius_schur_dense_error() < 1e-12


def test_mobius_schur_adjoint():
    assert pins.mobius_adjoint_error() < 1e-14


def test_shamir_gamma5_reflection_hermiticity():
    assert pins.shamir_reflection_error() < 1e-14


def test_cg_and_cgnr_vs_lapack():
    assert pins.cg_error() < 1e-11


def test_mobius_blocks_reassemble_full_operator():
    from oracle import domainwall

    dims, Ls = (4, 2, 2, 4), 5
    lat = Lattice(dims)
    op = domainwall.Mobius(synth.gauge_field(dims, 0.4, 93), lat, Ls, 1.8, 1.5, 0.5, 0.01)
    psi = synth.gaussian_spinor(dims, 93, nrhs=Ls)
    full = np.zeros_like(psi)
    for p in (0, 1):
        s = lat.sites_of(p)
        full[:, s] = op.D_pp(psi[:, s]) + op.D_hop(p, psi[:, lat.sites_of(1 - p)])
    assert pins.rel(full, op.full(psi)) < 1e-14


# --- staggered (Sec. 2 operators) --------------------------------------------------------


def test_staggered_free_field_normal_operator_closed_form():
    assert pins.staggered_free_field_error() < 1e-13


def test_staggered_hopping_antihermitian():
    assert pins.staggered_antihermitian_error() < 1e-15


def test_staggered_gauge_covariance():
    assert pins.staggered_covariance_error() < 1e-13


def test_staggered_dense_schur_and_evenodd_solve():
    assert pins.staggered_dense_error() < 1e-12


def test_staggered_phases():
    from oracle import staggered

    lat = Lattice((4, 2, 2, 2))
    c = lat.coords
    assert np.all(staggered.eta(lat, 0) == 1)
    assert np.all(staggered.eta(lat, 1) == (-1.0) ** c[0])
    assert np.all(staggered.eta(lat, 3) == (-1.0) ** (c[0] + c[1] + c[2]))


# --- two-level multigrid (Sec. 3) -------------------------------------------------------


def test_mg_transfer_operators():
    assert pins.mg_transfer_error() < 1e-13


def test_mg_coarse_operator_is_galerkin_and_g5_symmetric():
    assert pins.mg_coarse_error() < 1e-13


def test_mg_block_operator():
    assert pins.mg_block_operator_error() < 1e-14


def test_mg_sap_and_minimal_residual_step():
    assert pins.mg_sap_error() < 1e-12


def test_mg_cycle_composition():
    assert pins.mg_cycle_error() < 1e-12


def test_mg_fbicgstab_solve():
    assert pins.mg_solve_error() < 1e-10


def test_mg_coarse_evenodd_solve():
    assert pins.mg_coarse_evenodd_error() < 1e-10

