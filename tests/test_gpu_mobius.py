"""Moebius domain-wall operator and CG solve through the C-ABI against the oracle.

Operator parity element by element for D, D_eo, D_oe, the Schur operator of
Eq. 1 and its adjoint, in FP64 (1e-13) and FP32 (2e-6), on lattices with a
ragged last block of sites and fifth extents that leave idle threads in a
block (Ls = 1, 3, 5, 7, 16, 32).  Solves: against dense LU on a 2^4 lattice,
against the oracle's CG on the normal equations, a zero source among
several, and the mixed solve at the full 24^3 x 48 x 16 size with the
oracle's residual at sampled sites.
"""

import numpy as np
import pytest

import synth
from oracle import domainwall, solvers
from oracle.lattice import Lattice

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-13, "f32": 2e-6}
PARAMS = dict(M5=1.8, b5=1.5, c5=0.5, mf=0.01)


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def api():
    import __graft_entry__ as g

    g.build()
    from paper_2303_05883_gb300 import api

    return api


def _setup(api, dims, Ls, eps, seed, **kw):
    p = dict(PARAMS, **kw)
    lat = Lattice(dims)
    U = synth.gauge_field(dims, eps, seed)
    orc = domainwall.Mobius(U, lat, Ls, p["M5"], p["b5"], p["c5"], p["mf"])
    op = api.make_mobius(Ls, p["M5"], p["b5"], p["c5"], p["mf"])
    L = api.Lattice(dims)
    L.upload(U)
    return lat, U, orc, op, L


SHAPES = [((4, 4, 4, 8), 8), ((6, 4, 2, 4), 5), ((2, 2, 2, 2), 3), ((4, 2, 4, 6), 16), ((4, 4, 2, 2), 1),
          ((2, 4, 2, 4), 32), ((6, 6, 2, 4), 7)]


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("dims,Ls", SHAPES, ids=[f"{'x'.join(map(str, d))}_Ls{l}" for d, l in SHAPES])
def test_operators_match_oracle(api, dims, Ls, prec):
    lat, U, orc, op, L = _setup(api, dims, Ls, 0.4, 11 + Ls)
    nrhs = 2
    psi = synth.gaussian_spinor(dims, 7, nrhs=nrhs * Ls).reshape(nrhs, Ls, lat.V, 4, 3)
    got = L.D(op, psi, prec)
    for r in range(nrhs):
        assert rel(got[r], orc.full(psi[r])) < TOL[prec], ("D", r)
    # D_eo psi_o and D_oe psi_e
    for q in (0, 1):
        half = np.ascontiguousarray(psi[:, :, lat.sites_of(1 - q)])
        got = L.Deo(op, half, q, prec)
        for r in range(nrhs):
            assert rel(got[r], orc.D_hop(q, half[r])) < TOL[prec], ("Deo", q, r)
    xe = np.ascontiguousarray(psi[:, :, lat.even])
    got = L.Dhat(op, xe, prec)
    got_dag = L.Dhat_dag(op, xe, prec)
    for r in range(nrhs):
        assert rel(got[r], orc.schur(xe[r])) < TOL[prec], ("Dhat", r)
        assert rel(got_dag[r], orc.schur_dag(xe[r])) < TOL[prec], ("Dhat_dag", r)
    L.close()


def test_shamir_and_antiperiodic_x(api):
    """b = 1, c = 0 (Shamir) and a boundary phase in x as well."""
    dims, Ls = (4, 4, 2, 4), 6
    lat = Lattice(dims)
    U = synth.gauge_field(dims, 0.5, 3)
    bc = (-1, 1, 1, -1)
    orc = domainwall.Mobius(U, lat, Ls, 1.4, 1.0, 0.0, 0.2, bc=bc)
    op = api.make_mobius(Ls, 1.4, 1.0, 0.0, 0.2, bc=bc)
    L = api.Lattice(dims)
    L.upload(U)
    psi = synth.gaussian_spinor(dims, 9, nrhs=Ls)
    assert rel(L.D(op, psi, "f64"), orc.full(psi)) < 1e-13
    xe = np.ascontiguousarray(psi[:, lat.even])
    assert rel(L.Dhat(op, xe, "f32"), orc.schur(xe)) < 2e-6
    L.close()


def test_solve_matches_dense_lu(api):
    dims, Ls = (2, 2, 2, 2), 4
    lat, U, orc, op, L = _setup(api, dims, Ls, 0.5, 21, mf=0.05)
    b = synth.gaussian_spinor(dims, 22, nrhs=Ls)
    M = solvers.dense_matrix(lambda v: orc.full(v.reshape(Ls, lat.V, 4, 3)).reshape(-1), Ls * lat.V * 12)
    x_lu = np.linalg.solve(M, b.reshape(-1)).reshape(b.shape)
    for mixed, inner in ((1, "f32"), (0, "f64")):
        x, info = L.solve(op, b, api.make_solver(tol=1e-12, inner_prec=inner, mixed=mixed))
        assert info[0]["status"] == 0 and info[0]["true_rel_residual"] <= 1e-12, info
        assert rel(x, x_lu) < 1e-10, (mixed, rel(x, x_lu))
    L.close()


def test_solve_matches_oracle_cgnr_two_rhs_and_zero_source(api):
    dims, Ls = (4, 4, 4, 8), 8
    lat, U, orc, op, L = _setup(api, dims, Ls, 0.3, 31)
    b = synth.gaussian_spinor(dims, 32, nrhs=3 * Ls).reshape(3, Ls, lat.V, 4, 3)
    b[1] = 0.0  # a zero source between two others
    x, info = L.solve(op, b, api.make_solver(tol=1e-10, inner_prec="f32"))
    assert [i["status"] for i in info] == [0, 0, 0]
    assert np.abs(x[1]).max() == 0.0 and info[1]["true_rel_residual"] == 0.0
    for r in (0, 2):
        res = np.linalg.norm(b[r] - orc.full(x[r])) / np.linalg.norm(b[r])
        assert res <= 1.5e-10, res  # the oracle's own residual of the GPU solution
        assert info[r]["true_rel_residual"] <= 1e-10
    # the oracle's solution (CG on the normal equations to 1e-12) for one of them
    xe, oi = solvers.cgnr(orc.schur, orc.schur_dag, orc.prepare(b[0]), tol=1e-12)
    xo = orc.reconstruct(xe, b[0])
    assert rel(x[0], xo) < 5e-10, rel(x[0], xo)
    L.close()


def test_initial_guess_is_used(api):
    dims, Ls = (4, 2, 2, 4), 4
    lat, U, orc, op, L = _setup(api, dims, Ls, 0.3, 41)
    b = synth.gaussian_spinor(dims, 42, nrhs=Ls)
    x, info = L.solve(op, b, api.make_solver(tol=1e-11, inner_prec="f32"))
    x2, info2 = L.solve(op, b, api.make_solver(tol=1e-11, inner_prec="f32"), x0=x)
    assert info2[0]["status"] == 0 and info2[0]["inner_iters"] < info[0]["inner_iters"]
    assert rel(x2, x) < 1e-9
    L.close()


def test_rejected_arguments(api):
    from paper_2303_05883_gb300 import _abi

    dims = (4, 4, 2, 2)
    L = api.Lattice(dims)
    L.upload(synth.gauge_field(dims, 0.3, 1))
    psi = synth.gaussian_spinor(dims, 1, nrhs=4)
    with pytest.raises(_abi.BridgeError) as e:
        L.D(api.make_mobius(4, 1.8, 1.5, 0.5, 0.01), psi, "f16")
    assert e.value.status == _abi.BRIDGE_EINVAL
    with pytest.raises(_abi.BridgeError):
        L.D(api.make_mobius(0, 1.8, 1.5, 0.5, 0.01), psi[:1], "f64")
    with pytest.raises(_abi.BridgeError):
        L.D(api.make_mobius(33, 1.8, 1.5, 0.5, 0.01), np.zeros((33,) + psi.shape[1:], complex), "f64")
    # (b (4 - M5) + 1) = 0 and c (4 - M5) - 1 = 0 make D_ee singular
    with pytest.raises(_abi.BridgeError) as e:
        L.D(api.make_mobius(4, 5.0, 1.0, -1.0, 0.01), psi, "f64")
    assert e.value.status == _abi.BRIDGE_EINVAL
    with pytest.raises(_abi.BridgeError):
        L.Dhat_dag(api.make_op("wilson", 0.12), psi[0][::2].copy(), "f64")
    with pytest.raises(_abi.BridgeError):
        api.bridge_submit(L.handle, api.make_mobius(4, 1.8, 1.5, 0.5, 0.01), api.make_solver(), psi)
    L.close()


def _sample_sites(lat, n, seed):
    gen = np.random.default_rng(seed)
    L = lat.dims
    corners = [lat.index(np.array([[x], [y], [z], [t]]))[0]
               for x in (0, L[0] - 1) for y in (0, L[1] - 1) for z in (0, L[2] - 1) for t in (0, L[3] - 1)]
    return np.unique(np.concatenate([gen.choice(lat.V, n, replace=False), corners]))


def test_fullsize_24x24x24x48x16(api):
    """D at sampled sites in FP64 and FP32, then the mixed CG solve to 1e-10
    with the oracle's residual at sampled sites."""
    w = synth.WORKLOADS["mobius_24x24x24x48x16"]
    lat = Lattice(w.dims)
    U = w.gauge()
    orc = domainwall.Mobius(U, lat, w.Ls, w.M5, w.b5, w.c5, w.mf, w.bc)
    op = api.make_mobius(w.Ls, w.M5, w.b5, w.c5, w.mf, bc=w.bc)
    L = api.Lattice(w.dims)
    L.upload(U)
    b = w.sources()[0]
    s = _sample_sites(lat, 400, 1)
    want = orc.full(b, sites=s)
    for prec in ("f64", "f32"):
        got = L.D(op, b, prec)
        assert rel(got[:, s], want) < TOL[prec], prec
    del got
    x, info = L.solve(op, b, api.make_solver(tol=w.tol, inner_prec=w.inner))
    assert info[0]["status"] == 0 and info[0]["true_rel_residual"] <= w.tol, info
    r = b[:, s] - orc.full(x, sites=s)
    assert np.linalg.norm(r) / np.linalg.norm(b[:, s]) < 5 * w.tol
    L.close()


@pytest.mark.parametrize("how", ["env_dense", "unstable_recurrence"])
def test_dense_fifth_dimension_path(api, monkeypatch, how):
    """The dense s-matrix epilogue: forced by BRIDGE_DWF_DENSE, and chosen when
    |c(4-M5) - 1| > |b(4-M5) + 1| (the factored recurrence would grow)."""
    dims, Ls = (4, 2, 4, 4), 6
    if how == "env_dense":
        monkeypatch.setenv("BRIDGE_DWF_DENSE", "1")
        kw = {}
    else:
        kw = dict(b5=0.1, c5=1.5)
    lat, U, orc, op, L = _setup(api, dims, Ls, 0.4, 61, **kw)
    psi = synth.gaussian_spinor(dims, 62, nrhs=Ls)
    assert rel(L.D(op, psi, "f64"), orc.full(psi)) < 1e-13
    xe = np.ascontiguousarray(psi[:, lat.even])
    assert rel(L.Dhat(op, xe, "f32"), orc.schur(xe)) < 2e-6
    assert rel(L.Dhat_dag(op, xe, "f64"), orc.schur_dag(xe)) < 1e-13
    if how == "env_dense":  # (the other parameter set makes D_ee nearly singular: operators only)
        x, info = L.solve(op, psi, api.make_solver(tol=1e-10, inner_prec="f32"))
        assert info[0]["status"] == 0
        assert np.linalg.norm(psi - orc.full(x)) / np.linalg.norm(psi) < 1.5e-10
    L.close()


# every (fifth-dimension matrix, self term, epilogue) combination of the hop kernel
_DWF_COMBOS = [(1, 0, 0), (1, 1, 0), (1, 1, 1), (1, 1, 2), (1, 2, 0), (0, 0, 0), (0, 2, 0), (0, 2, 1)]


@pytest.mark.parametrize("block", [128, 256])
@pytest.mark.parametrize("variant", [3, 4, 5])
@pytest.mark.parametrize("dims,Ls", [((4, 2, 4, 6), 16), ((6, 6, 2, 4), 7), ((4, 4, 4, 8), 8)],
                         ids=["4x2x4x6_Ls16", "6x6x2x4_Ls7", "4x4x4x8_Ls8"])
def test_two_slices_per_thread_variants(api, dims, Ls, variant, block):
    """The hop kernels with two fifth-dimension slices per thread (links,
    neighbour indices and addresses shared by the slices s and s + Ls/2; a
    warp takes 16 sites x 2 slice groups, one or two such site tiles per
    block), pinned for every kernel of the operators and of the CG solve,
    against the oracle; an odd Ls runs the same variant with one slice per
    thread."""
    lat, U, orc, op, L = _setup(api, dims, Ls, 0.4, 40 + Ls)
    key = "x".join(map(str, dims))
    for nrhs in (1, 2):
        for m1, m2, epi in _DWF_COMBOS:
            api.bridge_tune_set(L.handle, f"dwf/1/{m1}/{m2}/{epi}/Ls{Ls}/{key}/{nrhs}", block, 1, variant)
    nrhs = 2
    psi = synth.gaussian_spinor(dims, 9, nrhs=nrhs * Ls).reshape(nrhs, Ls, lat.V, 4, 3)
    got = L.D(op, psi, "f32")
    for r in range(nrhs):
        assert rel(got[r], orc.full(psi[r])) < TOL["f32"], ("D", r)
    for q in (0, 1):
        half = np.ascontiguousarray(psi[:, :, lat.sites_of(1 - q)])
        got = L.Deo(op, half, q, "f32")
        for r in range(nrhs):
            assert rel(got[r], orc.D_hop(q, half[r])) < TOL["f32"], ("Deo", q, r)
    xe = np.ascontiguousarray(psi[:, :, lat.even])
    got, got_dag = L.Dhat(op, xe, "f32"), L.Dhat_dag(op, xe, "f32")
    for r in range(nrhs):
        assert rel(got[r], orc.schur(xe[r])) < TOL["f32"], ("Dhat", r)
        assert rel(got_dag[r], orc.schur_dag(xe[r])) < TOL["f32"], ("Dhat_dag", r)
    b = psi[0]
    x, info = L.solve(op, b, api.make_solver(tol=1e-10, inner_prec="f32"))
    assert info[0]["status"] == 0
    assert np.linalg.norm(b - orc.full(x)) / np.linalg.norm(b) <= 1.5e-10
    L.close()
