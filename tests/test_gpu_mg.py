"""Two-level multigrid through the C-ABI against the oracle.

With the null vectors passed in (seeded Gaussian vectors, the same on both
sides), the restriction, prolongation, coarse operator, SAP smoother and the
cycle are compared with oracle/multigrid.py; the FP32 preconditioner pieces
agree with the FP64 oracle to 2e-5.  The FBiCGStab solve (generated null
vectors) is compared with the oracle's solution / residual.
"""

import numpy as np
import pytest

import synth
from oracle import dirac, multigrid, solvers
from oracle.lattice import Lattice

pytestmark = pytest.mark.gpu

TOL32 = 2e-5


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def api():
    import __graft_entry__ as g

    g.build()
    from paper_2303_05883_gb300 import api

    return api


@pytest.fixture(scope="module")
def case(api):
    dims, block, nv, kappa, csw = (8, 8, 8, 8), (2, 2, 2, 2), 3, 0.12, 1.0
    lat = Lattice(dims)
    U = synth.gauge_field(dims, 0.3, 41)
    gen = np.random.default_rng(42)
    vs = gen.standard_normal((nv, lat.V, 4, 3)) + 1j * gen.standard_normal((nv, lat.V, 4, 3))
    orc = multigrid.Multigrid(U, lat, kappa, csw, block, vs)
    op = api.make_op("clover", kappa, csw)
    L = api.Lattice(dims)
    L.upload(U, op)
    # FP32 coarse operator in the coarse solver, so that the cycle can be
    # compared with the oracle's at a tight coarse tolerance
    mg = api.Multigrid(L, op, api.make_mg_params(block=block, nvec=nv, sap_cycles=2, mr_steps=4, coarse_tol=1e-6,
                                                 coarse_maxiter=1000, coarse_half=0), null_vectors=vs)
    yield dict(lat=lat, U=U, orc=orc, op=op, L=L, mg=mg, gen=gen)
    mg.close()
    L.close()


def test_restrict_and_prolong(api, case):
    from paper_2303_05883_gb300 import _abi

    orc, mg, gen, lat = case["orc"], case["mg"], case["gen"], case["lat"]
    v = gen.standard_normal((lat.V, 4, 3)) + 1j * gen.standard_normal((lat.V, 4, 3))
    assert rel(mg.apply(_abi.BRIDGE_MG_RESTRICT, v), orc.restrict(v)) < TOL32
    c = gen.standard_normal((mg.nblocks, 2, mg.nvec)) + 1j * gen.standard_normal((mg.nblocks, 2, mg.nvec))
    assert rel(mg.apply(_abi.BRIDGE_MG_PROLONG, c), orc.prolong(c)) < TOL32
    # P^dag P = 1 on the GPU's own basis
    assert rel(mg.apply(_abi.BRIDGE_MG_RESTRICT, mg.apply(_abi.BRIDGE_MG_PROLONG, c)), c) < TOL32


def test_coarse_operator_columns(api, case):
    """Columns of P^dag D P from the oracle against the GPU's nine couplings."""
    from paper_2303_05883_gb300 import _abi

    orc, mg, gen = case["orc"], case["mg"], case["gen"]
    G = mg.coarse_matrix()  # [X][d][col][row]
    nb, n2 = mg.nblocks, 2 * mg.nvec
    cd = orc.blocks.cdims

    def nbr(X, mu, step):
        c = list(np.unravel_index(X, cd[::-1])[::-1])
        c[mu] = (c[mu] + step) % cd[mu]
        return int(c[0] + cd[0] * (c[1] + cd[1] * (c[2] + cd[2] * c[3])))

    dense = np.zeros((nb * n2, nb * n2), dtype=np.complex128)
    for X in range(nb):
        for d in range(9):
            Y = X if d == 0 else nbr(X, (d - 1) // 2, -1 if (d - 1) % 2 else 1)
            dense[X * n2 : (X + 1) * n2, Y * n2 : (Y + 1) * n2] += G[X, d].T
    for col in gen.choice(nb * n2, 5, replace=False):
        e = np.zeros(nb * n2, dtype=np.complex128)
        e[col] = 1.0
        want = orc.restrict(orc.D(orc.prolong(e.reshape(nb, 2, mg.nvec)))).reshape(-1)
        assert rel(dense[:, col], want) < TOL32, col
    # the coarse operator application against the oracle's P^dag D P x
    x = gen.standard_normal((nb, 2, mg.nvec)) + 1j * gen.standard_normal((nb, 2, mg.nvec))
    assert rel(mg.apply(_abi.BRIDGE_MG_COARSE, x), orc.restrict(orc.D(orc.prolong(x)))) < TOL32


@pytest.mark.parametrize("nv", [3, 4, 12])
def test_coarse_operator_fp16_copy(api, case, nv):
    """The FP16 copy of D_c the coarse solver applies (tiled 16-byte rows for
    2 nv in 8, 16, 24, 32, 48; plain rows otherwise) against the oracle's
    P^dag D P x, within the FP16 rounding of the entries."""
    from paper_2303_05883_gb300 import _abi

    lat, U, op, L = case["lat"], case["U"], case["op"], case["L"]
    gen = np.random.default_rng(100 + nv)
    vs = gen.standard_normal((nv, lat.V, 4, 3)) + 1j * gen.standard_normal((nv, lat.V, 4, 3))
    orc = multigrid.Multigrid(U, lat, 0.12, 1.0, (2, 2, 2, 2), vs)
    mg = api.Multigrid(L, op, api.make_mg_params(block=(2, 2, 2, 2), nvec=nv, coarse_half=1), null_vectors=vs)
    x = gen.standard_normal((mg.nblocks, 2, nv)) + 1j * gen.standard_normal((mg.nblocks, 2, nv))
    want = orc.restrict(orc.D(orc.prolong(x)))
    assert rel(mg.apply(_abi.BRIDGE_MG_COARSE, x), want) < TOL32
    assert rel(mg.apply(_abi.BRIDGE_MG_COARSE_HALF, x), want) < 2e-3
    mg.close()
    # without the FP16 copy the half application is refused
    with pytest.raises(_abi.BridgeError):
        case["mg"].apply(_abi.BRIDGE_MG_COARSE_HALF, x[:, :, :3] if nv >= 3 else x)


@pytest.mark.parametrize("nv", [4, 12])
def test_coarse_solve_even_odd(api, case, nv):
    """The coarse BiCGStab on the FP16 copy, on the full coarse system and on
    its even-odd preconditioned form (with the odd part reconstructed), both
    against the oracle's P^dag D P: the residual is bounded by the FP16
    rounding of the coarse operator, and the two solutions agree."""
    from paper_2303_05883_gb300 import _abi

    lat, U, op, L = case["lat"], case["U"], case["op"], case["L"]
    gen = np.random.default_rng(200 + nv)
    vs = gen.standard_normal((nv, lat.V, 4, 3)) + 1j * gen.standard_normal((nv, lat.V, 4, 3))
    orc = multigrid.Multigrid(U, lat, 0.12, 1.0, (2, 2, 2, 2), vs)
    sols = []
    for eo in (0, 1):
        mg = api.Multigrid(L, op, api.make_mg_params(block=(2, 2, 2, 2), nvec=nv, coarse_half=1, coarse_eo=eo,
                                                     coarse_tol=1e-5, coarse_maxiter=4000), null_vectors=vs)
        r = np.random.default_rng(7).standard_normal((mg.nblocks, 2, nv)) + 0j
        e = mg.apply(_abi.BRIDGE_MG_COARSE_SOLVE, r)
        assert rel(orc.restrict(orc.D(orc.prolong(e))), r) < 2e-2, eo
        sols.append(e)
        mg.close()
    assert rel(sols[1], sols[0]) < 2e-2


@pytest.mark.parametrize("which", ["half", "solve"])
def test_coarse_wait_gives_up_and_reports(api, case, monkeypatch, which):
    """The bounded waits of the streamed coarse kernel.  With
    BRIDGE_MG_WAIT_POLLS=0 every site-loop wait gives up at once; nothing is
    faulted and no copy is lost (each CTA then waits, with the full bound, for
    the copies it still has in flight before it exits).  The kernel raises its
    error word and the call returns BRIDGE_ECUDA naming the wait; the next
    call on the same multigrid object, with the normal bound, succeeds (the
    word is cleared at the start of every coarse apply and solve) and agrees
    with the oracle."""
    from paper_2303_05883_gb300 import _abi

    lat, U, op, L = case["lat"], case["U"], case["op"], case["L"]
    nv = 4
    gen = np.random.default_rng(300)
    vs = gen.standard_normal((nv, lat.V, 4, 3)) + 1j * gen.standard_normal((nv, lat.V, 4, 3))
    orc = multigrid.Multigrid(U, lat, 0.12, 1.0, (2, 2, 2, 2), vs)
    mg = api.Multigrid(L, op, api.make_mg_params(block=(2, 2, 2, 2), nvec=nv, coarse_half=1, coarse_eo=1,
                                                 coarse_tol=1e-5, coarse_maxiter=4000), null_vectors=vs)
    x = gen.standard_normal((mg.nblocks, 2, nv)) + 1j * gen.standard_normal((mg.nblocks, 2, nv))
    op_id = _abi.BRIDGE_MG_COARSE_HALF if which == "half" else _abi.BRIDGE_MG_COARSE_SOLVE
    monkeypatch.setenv("BRIDGE_MG_WAIT_POLLS", "0")
    with pytest.raises(_abi.BridgeError) as e:
        mg.apply(op_id, x)
    assert e.value.status == _abi.BRIDGE_ECUDA
    assert "wait bound" in str(e.value) and "no longer reliable" not in str(e.value)
    monkeypatch.delenv("BRIDGE_MG_WAIT_POLLS")
    y = mg.apply(op_id, x)
    if which == "half":
        assert rel(y, orc.restrict(orc.D(orc.prolong(x)))) < 2e-3
    else:
        assert rel(orc.restrict(orc.D(orc.prolong(y))), x) < 2e-2
    mg.close()


def test_sap_smoother(api, case):
    from paper_2303_05883_gb300 import _abi

    orc, mg, gen, lat = case["orc"], case["mg"], case["gen"], case["lat"]
    r = gen.standard_normal((lat.V, 4, 3)) + 1j * gen.standard_normal((lat.V, 4, 3))
    assert rel(mg.apply(_abi.BRIDGE_MG_SAP, r), orc.sap(r, 2, 4)) < TOL32


@pytest.mark.parametrize("fused", ["1", "0"])
def test_sap_residual_inside_sweep_or_separate(api, monkeypatch, fused):
    """The SAP sweep with the block residual r - D x formed inside the sweep
    kernel (default) and with the separate residual pass, on 4x2x2x2 blocks
    with a negative phase in y and t, against the oracle's smoother (three
    cycles: every half sweep after the first forms its residual from a
    nonzero x)."""
    from paper_2303_05883_gb300 import _abi

    dims, block, nv, kappa, csw, bc = (8, 4, 4, 8), (4, 2, 2, 2), 2, 0.115, 1.0, (1, -1, 1, -1)
    lat = Lattice(dims)
    U = synth.gauge_field(dims, 0.35, 77)
    gen = np.random.default_rng(78)
    vs = gen.standard_normal((nv, lat.V, 4, 3)) + 1j * gen.standard_normal((nv, lat.V, 4, 3))
    orc = multigrid.Multigrid(U, lat, kappa, csw, block, vs, bc=bc)
    op = api.make_op("clover", kappa, csw, bc)
    L = api.Lattice(dims)
    L.upload(U, op)
    monkeypatch.setenv("BRIDGE_MG_SAP_FUSED", fused)
    mg = api.Multigrid(L, op, api.make_mg_params(block=block, nvec=nv, sap_cycles=3, mr_steps=5, coarse_half=0),
                       null_vectors=vs)
    monkeypatch.delenv("BRIDGE_MG_SAP_FUSED")
    r = gen.standard_normal((lat.V, 4, 3)) + 1j * gen.standard_normal((lat.V, 4, 3))
    assert rel(mg.apply(_abi.BRIDGE_MG_SAP, r), orc.sap(r, 3, 5)) < TOL32
    mg.close()
    L.close()


def test_cycle(api, case):
    """The preconditioner with a tight coarse tolerance against the oracle's
    cycle with a tight coarse BiCGStab."""
    from paper_2303_05883_gb300 import _abi

    orc, mg, gen, lat = case["orc"], case["mg"], case["gen"], case["lat"]
    r = gen.standard_normal((lat.V, 4, 3)) + 1j * gen.standard_normal((lat.V, 4, 3))

    def coarse(rc):
        A = lambda v: orc.restrict(orc.D(orc.prolong(v.reshape(rc.shape)))).reshape(-1)  # noqa: E731
        x, _ = solvers.bicgstab(A, rc.reshape(-1), tol=1e-9, maxiter=5000)
        return x.reshape(rc.shape)

    want = orc.cycle(r, 2, 4, coarse_solve=coarse)
    assert rel(mg.apply(_abi.BRIDGE_MG_CYCLE, r), want) < 1e-4


def test_solve_matches_oracle(api, case):
    """FBiCGStab with the two-level preconditioner reaches the oracle's solution."""
    lat, U, op, L = case["lat"], case["U"], case["op"], case["L"]
    b = synth.gaussian_spinor(lat.dims, 43)
    mg = api.Multigrid(L, op, api.make_mg_params(block=(2, 2, 2, 2), nvec=6))
    x, info = mg.solve(b, api.make_solver(tol=1e-12, max_iter=200))
    mg.close()
    assert info[0]["status"] == 0 and info[0]["true_rel_residual"] <= 1e-12
    T = dirac.clover_term(U, lat, 0.12, 1.0)
    xo, _ = solvers.bicgstab(lambda v: dirac.dirac(U, v, lat, 0.12, 1.0, T=T), b, tol=1e-13)
    assert rel(x, xo) < 1e-10


def test_solve_16x16x16x32_generated_null_space(api):
    dims = (16, 16, 16, 32)
    lat = Lattice(dims)
    U = synth.gauge_field(dims, 0.2, 44)
    kappa, csw = 0.124, 1.0
    op = api.make_op("clover", kappa, csw)
    L = api.Lattice(dims)
    L.upload(U, op)
    b = synth.gaussian_spinor(dims, 45)
    mg = api.Multigrid(L, op, api.make_mg_params(nvec=12))
    x, info = mg.solve(b, api.make_solver(tol=1e-10, max_iter=500))
    assert info[0]["status"] == 0 and info[0]["true_rel_residual"] <= 1e-10, info
    s = np.random.default_rng(1).choice(lat.V, 2000, replace=False)
    r = b[s] - dirac.dirac(U, x, lat, kappa, csw, sites=s)
    assert np.linalg.norm(r) / np.linalg.norm(b[s]) < 5e-10
    # the same system by the mixed BiCGStab takes far more operator applications
    _, info2 = L.solve(op, b, api.make_solver(tol=1e-10))
    assert info[0]["inner_iters"] < info2[0]["inner_iters"]
    mg.close()
    L.close()


def test_rejected_parameters(api):
    from paper_2303_05883_gb300 import _abi

    dims = (8, 8, 8, 8)
    L = api.Lattice(dims)
    op = api.make_op("clover", 0.12, 1.0)
    with pytest.raises(_abi.BridgeError):  # no gauge field yet
        api.Multigrid(L, op)
    L.upload(synth.gauge_field(dims, 0.3, 1), op)
    for kw in (dict(block=(3, 2, 2, 2)), dict(block=(8, 2, 2, 2)), dict(nvec=0), dict(nvec=40)):
        with pytest.raises(_abi.BridgeError):
            api.Multigrid(L, op, api.make_mg_params(**kw))
    with pytest.raises(_abi.BridgeError):
        api.Multigrid(L, api.make_mobius(4, 1.8, 1.5, 0.5, 0.1))
    L.close()
