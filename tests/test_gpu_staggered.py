"""Staggered operator and CG solve through the C-ABI against the oracle.

Operator parity element by element for D, D_eo, D_oe and the Schur operator
of Eq. 1 in FP64 (1e-13) and FP32 (2e-6) on lattices with ragged last
blocks; solves against dense LU and the oracle's CG, a zero source among
several, an initial guess; the full 64^4 FP32 / FP64 solve with the
oracle's residual at sampled sites.
"""

import numpy as np
import pytest

import synth
from oracle import solvers, staggered
from oracle.lattice import Lattice
from tests import pins

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-13, "f32": 2e-6}


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def api():
    import __graft_entry__ as g

    g.build()
    from paper_2303_05883_gb300 import api

    return api


def _vec(lat, seed, n=None):
    gen = np.random.default_rng(seed)
    shape = (lat.V, 3) if n is None else (n, lat.V, 3)
    return gen.standard_normal(shape) + 1j * gen.standard_normal(shape)


SHAPES = [(4, 4, 4, 8), (6, 4, 2, 4), (2, 2, 2, 2), (8, 6, 4, 2), (10, 2, 2, 6)]


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("dims", SHAPES, ids=["x".join(map(str, d)) for d in SHAPES])
def test_operators_match_oracle(api, dims, prec):
    lat = Lattice(dims)
    U = synth.gauge_field(dims, 0.4, 5)
    bc = (1, -1, 1, -1)
    orc = staggered.Staggered(U, lat, 0.07, bc)
    op = api.make_staggered(0.07, bc=bc)
    L = api.Lattice(dims)
    L.upload(U)
    chi = _vec(lat, 1, n=2)
    got = L.D(op, chi, prec)
    for r in range(2):
        assert rel(got[r], orc.full(chi[r])) < TOL[prec], ("D", r)
    for q in (0, 1):
        half = np.ascontiguousarray(chi[:, lat.sites_of(1 - q)])
        got = L.Deo(op, half, q, prec)
        for r in range(2):
            assert rel(got[r], orc.D_hop(q, half[r])) < TOL[prec], ("Deo", q, r)
    xe = np.ascontiguousarray(chi[:, lat.even])
    got = L.Dhat(op, xe, prec)
    for r in range(2):
        assert rel(got[r], orc.schur(xe[r])) < TOL[prec], ("Dhat", r)
    L.close()


def test_solve_matches_dense_lu(api):
    dims, m = (2, 2, 2, 4), 0.1
    lat = Lattice(dims)
    U = synth.gauge_field(dims, 0.5, 7)
    M = pins.dense_staggered(U, lat, m)
    b = _vec(lat, 8)
    x_lu = np.linalg.solve(M, b.reshape(-1)).reshape(b.shape)
    L = api.Lattice(dims)
    L.upload(U)
    op = api.make_staggered(m)
    for mixed, inner in ((1, "f32"), (0, "f64")):
        x, info = L.solve(op, b, api.make_solver(tol=1e-12, inner_prec=inner, mixed=mixed))
        assert info[0]["status"] == 0 and info[0]["true_rel_residual"] <= 1e-12, info
        assert rel(x, x_lu) < 1e-10, (mixed, rel(x, x_lu))
    L.close()


def test_solve_matches_oracle_cg_with_zero_source(api):
    dims, m = (4, 4, 4, 8), 0.05
    lat = Lattice(dims)
    U = synth.gauge_field(dims, 0.3, 9)
    orc = staggered.Staggered(U, lat, m)
    b = _vec(lat, 10, n=3)
    b[1] = 0.0
    L = api.Lattice(dims)
    L.upload(U)
    x, info = L.solve(api.make_staggered(m), b, api.make_solver(tol=1e-10, inner_prec="f32"))
    assert [i["status"] for i in info] == [0, 0, 0]
    assert np.abs(x[1]).max() == 0.0
    for r in (0, 2):
        assert np.linalg.norm(b[r] - orc.full(x[r])) / np.linalg.norm(b[r]) <= 1.5e-10
    xe, _ = solvers.cg(orc.normal_even, orc.prepare(b[0]), tol=1e-13)
    assert rel(x[0], orc.reconstruct(xe, b[0])) < 5e-10
    # an initial guess at the solution needs no iterations
    x2, info2 = L.solve(api.make_staggered(m), b[0], api.make_solver(tol=1e-10, inner_prec="f32"), x0=x[0])
    assert info2[0]["status"] == 0 and info2[0]["inner_iters"] == 0
    L.close()


def test_rejected_arguments(api):
    from paper_2303_05883_gb300 import _abi

    dims = (4, 4, 2, 2)
    lat = Lattice(dims)
    L = api.Lattice(dims)
    L.upload(synth.gauge_field(dims, 0.3, 1))
    chi = _vec(lat, 2)
    with pytest.raises(_abi.BridgeError):
        L.D(api.make_staggered(0.0), chi, "f64")
    with pytest.raises(_abi.BridgeError):
        L.D(api.make_staggered(0.1), chi, "bf16")
    with pytest.raises(_abi.BridgeError):
        L.Dhat_dag(api.make_staggered(0.1), chi[lat.even], "f64")
    with pytest.raises(_abi.BridgeError):
        api.bridge_submit(L.handle, api.make_staggered(0.1), api.make_solver(), chi)
    L.close()


def test_fullsize_64x64x64x64(api):
    """D at sampled sites (FP64, FP32), then the mixed solve to 1e-10 with the
    oracle's residual at sampled sites."""
    w = synth.WORKLOADS["staggered_64x64x64x64"]
    lat = Lattice(w.dims)
    U = w.gauge()
    orc = staggered.Staggered(U, lat, w.mass, w.bc)
    op = api.make_staggered(w.mass, bc=w.bc)
    L = api.Lattice(w.dims)
    L.upload(U)
    b = w.sources()[0]
    gen = np.random.default_rng(3)
    s = np.unique(np.concatenate([gen.choice(lat.V, 3000, replace=False), [0, lat.V - 1]]))
    want = orc.full(b, sites=s)
    for prec in ("f64", "f32"):
        assert rel(L.D(op, b, prec)[s], want) < TOL[prec], prec
    x, info = L.solve(op, b, api.make_solver(tol=w.tol, inner_prec=w.inner))
    assert info[0]["status"] == 0 and info[0]["true_rel_residual"] <= w.tol, info
    r = b[s] - orc.full(x, sites=s)
    assert np.linalg.norm(r) / np.linalg.norm(b[s]) < 5 * w.tol
    L.close()
