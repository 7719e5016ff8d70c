"""GPU solves against the FP64 oracle.

Every solver configuration (plain FP64 BiCGStab; FP32, FP16 and BF16 inner
solvers inside the FP64 defect-correction loop) must return x within 1e-10
relative L2 of the oracle's solution of D x = b, with the oracle solved to a
residual tight enough that its own error is far below that bar.  Edge cases:
zero sources, an exact initial guess, iteration limits, 12 point sources,
graph replay vs direct launches.
"""

import numpy as np
import pytest

import synth
from oracle import dirac, evenodd, solvers
from oracle.lattice import Lattice

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def api():
    import __graft_entry__ as g

    g.build()
    from paper_2303_05883_gb300 import api

    return api


def oracle_solve(U, lat, kappa, csw, b, bc=(1, 1, 1, -1), tol=1e-14):
    eo = evenodd.EvenOdd(U, lat, kappa, csw, bc)
    xe, info = solvers.bicgstab(eo.schur, eo.prepare(b), tol=tol)
    x = eo.reconstruct(xe, b)
    T = dirac.clover_term(U, lat, kappa, csw)
    r = b - dirac.dirac(U, x, lat, kappa, csw, bc, T=T)
    return x, float(np.linalg.norm(r) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def wilson8(api):
    """8^4 Wilson, kappa 0.12, links exp(0.3 i A), Gaussian source (seed 1)."""
    w = synth.WORKLOADS["wilson_8x8x8x8"]
    lat = Lattice(w.dims)
    U = w.gauge()
    b = w.sources()[0]
    x, res = oracle_solve(U, lat, w.kappa, 0.0, b)
    assert res < 1e-13
    L = api.Lattice(w.dims)
    op = api.make_op("wilson", w.kappa)
    L.upload(U, op)
    yield dict(L=L, op=op, U=U, b=b, x=x, lat=lat, w=w)
    L.close()


@pytest.fixture(scope="module")
def clover_odd(api):
    """Non-cubic clover case with a ragged last thread block."""
    dims, kappa, csw = (4, 6, 8, 10), 0.125, 1.0
    lat = Lattice(dims)
    U = synth.gauge_field(dims, 0.2, 7)
    b = synth.gaussian_spinor(dims, 7)
    x, res = oracle_solve(U, lat, kappa, csw, b)
    assert res < 1e-13
    L = api.Lattice(dims)
    op = api.make_op("clover", kappa, csw)
    L.upload(U, op)
    yield dict(L=L, op=op, U=U, b=b, x=x, lat=lat, kappa=kappa, csw=csw)
    L.close()


@pytest.mark.parametrize(
    "mode", [dict(mixed=0), dict(mixed=1, inner_prec="f32"), dict(mixed=1, inner_prec="f16"), dict(mixed=1, inner_prec="bf16")]
)
def test_wilson_8x8x8x8_solve(wilson8, api, mode):
    s = api.make_solver(tol=1e-12, **mode)
    x, info = wilson8["L"].solve(wilson8["op"], wilson8["b"], s)
    assert info[0]["status"] == 0
    assert info[0]["true_rel_residual"] <= 1e-12
    assert rel(x, wilson8["x"]) < 1e-10


@pytest.mark.parametrize(
    "mode", [dict(mixed=0), dict(mixed=1, inner_prec="f32"), dict(mixed=1, inner_prec="f16"), dict(mixed=1, inner_prec="bf16")]
)
def test_clover_noncubic_solve(clover_odd, api, mode):
    s = api.make_solver(tol=1e-12, **mode)
    x, info = clover_odd["L"].solve(clover_odd["op"], clover_odd["b"], s)
    assert info[0]["status"] == 0 and info[0]["true_rel_residual"] <= 1e-12
    assert rel(x, clover_odd["x"]) < 1e-10


def test_dense_lu_2x2x2x2(api):
    dims, kappa, csw = (2, 2, 2, 2), 0.12, 1.0
    lat = Lattice(dims)
    U = synth.gauge_field(dims, 0.5, 51)
    b = synth.gaussian_spinor(dims, 51)
    M = solvers.dense_dirac(U, lat, kappa, csw)
    x_lu = solvers.lu_solve(M, b.reshape(-1)).reshape(b.shape)
    L = api.Lattice(dims)
    op = api.make_op("clover", kappa, csw)
    L.upload(U, op)
    for mode in (dict(mixed=0), dict(mixed=1, inner_prec="f32")):
        x, info = L.solve(op, b, api.make_solver(tol=1e-13, **mode))
        assert rel(x, x_lu) < 1e-11
    L.close()


def test_free_field_inverse_on_gpu(api):
    from tests import pins

    dims, kappa = (4, 4, 4, 8), 0.12
    lat = Lattice(dims)
    gen = np.random.default_rng(3)
    u = gen.standard_normal((4, 3)) + 1j * gen.standard_normal((4, 3))
    b, p = pins.plane_wave(lat, (1, 0, 2, 3), u)
    want = np.einsum("st,ntc->nsc", np.linalg.inv(pins.free_field_symbol(p, kappa)), b)
    L = api.Lattice(dims)
    op = api.make_op("wilson", kappa)
    L.upload(synth.unit_gauge(dims), op)
    x, info = L.solve(op, b, api.make_solver(tol=1e-13))
    assert rel(x, want) < 1e-11
    L.close()


def test_twelve_point_sources_f16(api):
    """12 spin-colour point sources at the origin, FP16 inner solver, all at once."""
    dims, kappa, csw = (4, 4, 4, 8), 0.125, 1.0
    lat = Lattice(dims)
    U = synth.gauge_field(dims, 0.2, 3)
    B = synth.point_sources(dims)
    eo = evenodd.EvenOdd(U, lat, kappa, csw)
    L = api.Lattice(dims)
    op = api.make_op("clover", kappa, csw)
    L.upload(U, op)
    X, info = L.solve(op, B, api.make_solver(tol=1e-12, inner_prec="f16"))
    assert len(info) == 12
    for k in range(12):
        xe, _ = solvers.bicgstab(eo.schur, eo.prepare(B[k]), tol=1e-14)
        xk = eo.reconstruct(xe, B[k])
        assert info[k]["status"] == 0 and info[k]["true_rel_residual"] <= 1e-12
        assert rel(X[k], xk) < 1e-10, k
    L.close()


def test_multi_rhs_equals_single_rhs(clover_odd, api):
    """Right-hand sides solved together give the same answer as alone (within the bar)."""
    b2 = np.stack([clover_odd["b"], synth.gaussian_spinor((4, 6, 8, 10), 8)])
    s = api.make_solver(tol=1e-12)
    X, info = clover_odd["L"].solve(clover_odd["op"], b2, s)
    x0, _ = clover_odd["L"].solve(clover_odd["op"], b2[0], s)
    assert rel(X[0], x0) < 1e-10 and rel(X[0], clover_odd["x"]) < 1e-10


def test_zero_source_and_zero_column(clover_odd, api):
    s = api.make_solver(tol=1e-12)
    z = np.zeros_like(clover_odd["b"])
    guess = synth.gaussian_spinor((4, 6, 8, 10), 9)
    x, info = clover_odd["L"].solve(clover_odd["op"], z, s, x0=guess)
    assert np.abs(x).max() == 0 and info[0]["status"] == 0
    B = np.stack([z, clover_odd["b"]])
    X, info = clover_odd["L"].solve(clover_odd["op"], B, s)
    assert np.abs(X[0]).max() == 0 and rel(X[1], clover_odd["x"]) < 1e-10


def test_exact_initial_guess_needs_no_iterations(clover_odd, api):
    s = api.make_solver(tol=1e-10)
    x, info = clover_odd["L"].solve(clover_odd["op"], clover_odd["b"], s, x0=clover_odd["x"])
    assert info[0]["inner_iters"] == 0 and info[0]["true_rel_residual"] <= 1e-10


def test_iteration_limit_reports_enoconv(clover_odd, api):
    from paper_2303_05883_gb300 import _abi

    s = api.make_solver(tol=1e-12, max_iter=3, check_every=1)
    x, info = clover_odd["L"].solve(clover_odd["op"], clover_odd["b"], s, raise_on_fail=False)
    assert info[0]["status"] == _abi.BRIDGE_ENOCONV
    assert info[0]["true_rel_residual"] > 1e-12


def test_graph_replay_is_bit_identical_to_direct_launches(clover_odd, api):
    a, _ = clover_odd["L"].solve(clover_odd["op"], clover_odd["b"], api.make_solver(tol=1e-11, use_graph=1))
    b, _ = clover_odd["L"].solve(clover_odd["op"], clover_odd["b"], api.make_solver(tol=1e-11, use_graph=0))
    assert np.array_equal(a, b)


def test_repeat_solve_is_bit_identical(clover_odd, api):
    s = api.make_solver(tol=1e-11, inner_prec="f16")
    a, _ = clover_odd["L"].solve(clover_odd["op"], clover_odd["b"], s)
    b, _ = clover_odd["L"].solve(clover_odd["op"], clover_odd["b"], s)
    assert np.array_equal(a, b)


def test_profile_stats_report_event_times(clover_odd, api):
    h = clover_odd["L"].handle
    api.bridge_stats_reset(h)
    api.bridge_profile(h, True)
    clover_odd["L"].solve(clover_odd["op"], clover_odd["b"], api.make_solver(tol=1e-10))
    api.bridge_profile(h, False)
    st = api.bridge_stats(h)
    assert st["schur_pass2_alpha"]["launches"] > 0 and st["schur_pass2_alpha"]["ms"] > 0
    assert st["schur_pass2_omega"]["launches"] == st["schur_pass2_alpha"]["launches"]
    assert st["residual64"]["launches"] >= 4


def test_autotuned_shapes_keep_parity(clover_odd, api):
    """Autotuning changes launch shapes (and reduction order) but not the answer."""
    h = clover_odd["L"].handle
    api.bridge_tune(h, clover_odd["op"], "f32", 1)
    table = api.bridge_tune_table(h)
    assert any(k.startswith("hop/1/") for k in table) and any(k.startswith("blas/") for k in table)
    for block, nblk, variant in table.values():
        assert block in (64, 128, 256) and nblk >= 1 and 0 <= variant < 6
    x, info = clover_odd["L"].solve(clover_odd["op"], clover_odd["b"], api.make_solver(tol=1e-12))
    assert info[0]["true_rel_residual"] <= 1e-12 and rel(x, clover_odd["x"]) < 1e-10


@pytest.mark.parametrize("prec", ["f32", "f16"])
@pytest.mark.parametrize("variant", [3, 5, 6, 7, 8, 9, 10, 11, 12])
def test_forced_kernel_variants_keep_parity(api, prec, variant):
    """Every stencil variant (read-once loads, 2/3/4 right-hand sides per
    thread, the shared-link tile kernel with and without pipelined
    neighbour loads) inside a 5-RHS solve -- ragged
    right-hand-side groups -- against
    the oracle, with the launch shape pinned by bridge_tune_set."""
    dims, kappa, csw, nrhs = (4, 6, 8, 10), 0.125, 1.0, 5
    lat = Lattice(dims)
    U = synth.gauge_field(dims, 0.2, 17)
    B = synth.gaussian_spinor(dims, 17, nrhs=nrhs)
    L = api.Lattice(dims)
    op = api.make_op("clover", kappa, csw)
    L.upload(U, op)
    p = {"f32": 1, "f16": 2}[prec]
    key = "x".join(map(str, dims))
    for flags, red in [(4, 0), (5, 2), (5, 3), (0, 0)]:
        api.bridge_tune_set(L.handle, f"hop/{p}/{flags}/{red}/{key}/{nrhs}", 64, 3, variant)
    X, info = L.solve(op, B, api.make_solver(tol=1e-12, inner_prec=prec))
    eo = evenodd.EvenOdd(U, lat, kappa, csw)
    for k in range(nrhs):
        xe, _ = solvers.bicgstab(eo.schur, eo.prepare(B[k]), tol=1e-14)
        assert info[k]["status"] == 0 and rel(X[k], eo.reconstruct(xe, B[k])) < 1e-10, (k, info[k])
    # D_eo with the same pinned variant, against the oracle block
    got = L.Deo(op, np.ascontiguousarray(B[:, lat.odd]), 0, prec)
    want = np.stack([eo.D_hop(0, B[k][lat.odd]) for k in range(nrhs)])
    assert rel(got, want) < {"f32": 2e-6, "f16": 5e-3}[prec]
    L.close()


def test_nonfinite_source_reports_breakdown(clover_odd, api):
    """A NaN in b propagates to the FP64 residual; the solve stops with EBREAKDOWN."""
    from paper_2303_05883_gb300 import _abi

    b = clover_odd["b"].copy()
    b[7, 1, 2] = np.nan
    x, info = clover_odd["L"].solve(clover_odd["op"], b, api.make_solver(tol=1e-10), raise_on_fail=False)
    assert info[0]["status"] == _abi.BRIDGE_EBREAKDOWN
    # the lattice stays usable
    x, info = clover_odd["L"].solve(clover_odd["op"], clover_odd["b"], api.make_solver(tol=1e-12))
    assert info[0]["status"] == 0 and rel(x, clover_odd["x"]) < 1e-10


def test_null_pointers_are_einval(clover_odd, api):
    import ctypes

    from paper_2303_05883_gb300 import _abi

    lib = _abi.load()
    op = clover_odd["op"]
    h = clover_odd["L"].handle
    assert lib.bridge_mult_D(h, ctypes.byref(op), 1, None, None, 1) == _abi.BRIDGE_EINVAL
    assert lib.bridge_mult_D(h, None, 1, None, None, 1) == _abi.BRIDGE_EINVAL
    s = api.make_solver()
    assert lib.bridge_solve(h, ctypes.byref(op), ctypes.byref(s), None, None, 1, None) == _abi.BRIDGE_EINVAL
    assert lib.bridge_gauge_upload(h, None, None) == _abi.BRIDGE_EINVAL
    assert lib.bridge_apply(h, ctypes.byref(op), 9, None, None) == _abi.BRIDGE_EINVAL


def test_alu_peak_is_measured(api):
    """The FMA microbenchmark behind the arithmetic rooflines: FP32 well above
    FP64 (the FP64 pipe runs at a small fraction of the FP32 rate) and both
    within physical bounds (152 SMs x 128 FP32 lanes x 2 flops x 2.1 GHz)."""
    f32, f64 = api.bridge_alu_peak("f32"), api.bridge_alu_peak("f64")
    assert 1e12 < f32 < 1.2e14
    assert 1e10 < f64 < f32 / 4


@pytest.mark.parametrize("kind,prec", [("clover", "f64"), ("clover", "f32"), ("wilson", "f32"), ("clover", "f16")])
def test_cgnr_inner_method_matches_oracle(api, kind, prec):
    """CG on the normal equations of the Schur system (the inner method the
    solver switches to where BiCGStab stagnates), forced for every pass, on a
    lattice with several site blocks: the solution agrees with the oracle's
    even-odd BiCGStab solution of the same system."""
    from paper_2303_05883_gb300 import _abi

    dims, kappa, nrhs = (4, 6, 8, 10), 0.125, 2
    csw = 1.0 if kind == "clover" else 0.0
    lat = Lattice(dims)
    U = synth.gauge_field(dims, 0.3, 23)
    B = synth.gaussian_spinor(dims, 23, nrhs=nrhs)
    L = api.Lattice(dims)
    op = api.make_op(kind, kappa, csw)
    L.upload(U, op)
    X, info = L.solve(op, B, api.make_solver(tol=1e-11, inner_prec=prec, method=_abi.BRIDGE_METHOD_CGNR,
                                             max_iter=40000))
    eo = evenodd.EvenOdd(U, lat, kappa, csw)
    for k in range(nrhs):
        xe, _ = solvers.bicgstab(eo.schur, eo.prepare(B[k]), tol=1e-14)
        assert info[k]["status"] == 0 and info[k]["cgnr_passes"] == info[k]["outer_iters"], info[k]
        assert rel(X[k], eo.reconstruct(xe, B[k])) < 1e-9, (k, rel(X[k], eo.reconstruct(xe, B[k])))
    L.close()


def test_auto_method_switches_to_cgnr_past_critical_kappa(api):
    """kappa = 0.15 on a smooth field (links exp(0.1 i A)) is far past the
    critical kappa: the eigenvalues of D surround the origin and BiCGStab
    stagnates (alone it ends at the iteration limit), while D^dag D stays well
    conditioned.  The automatic method switches to CG on the normal equations
    after one stagnating BiCGStab pass and meets the tolerance; the oracle's
    residual b - D x over the whole lattice confirms it."""
    from paper_2303_05883_gb300 import _abi

    dims, kappa = (8, 8, 8, 8), 0.15
    lat = Lattice(dims)
    U = synth.gauge_field(dims, 0.1, 11)
    b = synth.gaussian_spinor(dims, 5)
    L = api.Lattice(dims)
    op = api.make_op("wilson", kappa)
    L.upload(U, op)
    _, info = L.solve(op, b, api.make_solver(tol=1e-10, method=_abi.BRIDGE_METHOD_BICGSTAB, max_iter=4000),
                      raise_on_fail=False)
    assert info[0]["status"] == _abi.BRIDGE_ENOCONV and info[0]["cgnr_passes"] == 0
    x, info = L.solve(op, b, api.make_solver(tol=1e-10, max_iter=40000))
    assert info[0]["status"] == 0 and info[0]["cgnr_passes"] >= 1, info[0]
    assert info[0]["true_rel_residual"] <= 1e-10
    r = b - dirac.dirac(U, x, lat, kappa, 0.0)
    assert np.linalg.norm(r) / np.linalg.norm(b) < 2e-10
    L.close()
