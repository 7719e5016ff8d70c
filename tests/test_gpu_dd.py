"""The lattice decomposed into slabs along t with a halo exchange, against the
FP64 oracle on the whole lattice.

Two and four slabs on one GPU: the full operator, D_eo, D_oe and the Schur
operator of Eq. 1 in every storage precision, and the decomposed BiCGStab
solve.  Every slab boundary (and the lattice boundary with its antiperiodic
phase) is crossed by t hops, so a wrong face, index or phase fails the
element-wise comparison; the per-site maximum error is bounded as well as
the relative L2 error.
"""

import numpy as np
import pytest

import synth
from oracle import evenodd, solvers
from oracle.lattice import Lattice

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-13, "f32": 2e-6, "f16": 5e-3, "bf16": 5e-3}


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def site_max(a, b):
    e = np.linalg.norm((a - b).reshape(a.shape[0], a.shape[1], -1), axis=2)
    n = np.linalg.norm(b.reshape(b.shape[0], b.shape[1], -1), axis=2)
    return float(e.max() / np.sqrt(np.mean(n ** 2)))


@pytest.fixture(scope="module")
def api():
    import __graft_entry__ as g

    g.build()
    from paper_2303_05883_gb300 import api

    return api


CASES = [
    # dims, kind, kappa, csw, bc, nrhs
    ((4, 6, 4, 8), "clover", 0.125, 1.0, (1, 1, 1, -1), 2),
    ((6, 4, 4, 8), "wilson", 0.12, 0.0, (1, -1, 1, -1), 1),
    ((8, 8, 8, 16), "clover", 0.125, 1.0, (1, 1, 1, -1), 1),
]


@pytest.fixture(scope="module", params=range(len(CASES)), ids=lambda i: "x".join(map(str, CASES[i][0])) + "-" + CASES[i][1])
def case(request, api):
    dims, kind, kappa, csw, bc, nrhs = CASES[request.param]
    lat = Lattice(dims)
    U = synth.gauge_field(dims, 0.4, 60 + request.param)
    psi = synth.gaussian_spinor(dims, 60 + request.param, nrhs=nrhs)
    eo = evenodd.EvenOdd(U, lat, kappa, csw, bc)
    op = api.make_op(kind, kappa, csw, bc)
    L = api.Lattice(dims)
    L.upload(U, op)
    want = {
        "D": np.stack([eo.full(p) for p in psi]),
        "Deo": np.stack([eo.D_hop(0, p[lat.odd]) for p in psi]),
        "Doe": np.stack([eo.D_hop(1, p[lat.even]) for p in psi]),
        "Dhat": np.stack([eo.schur(p[lat.even]) for p in psi]),
    }
    yield dict(lat=lat, U=U, psi=psi, eo=eo, op=op, L=L, want=want, kappa=kappa, csw=csw, bc=bc)
    L.close()


@pytest.mark.parametrize("nparts", [2, 4])
@pytest.mark.parametrize("prec", ["f64", "f32", "f16", "bf16"])
def test_decomposed_operators(api, case, nparts, prec):
    lat, psi = case["lat"], case["psi"]
    if lat.dims[3] % (2 * nparts):
        pytest.skip("slabs of an odd number of time slices")
    dd = api.Decomposition(case["L"], case["op"], nparts)
    got = {
        "D": dd.D(psi, prec),
        "Deo": dd.Deo(np.ascontiguousarray(psi[:, lat.odd]), 0, prec),
        "Doe": dd.Deo(np.ascontiguousarray(psi[:, lat.even]), 1, prec),
        "Dhat": dd.Dhat(np.ascontiguousarray(psi[:, lat.even]), prec),
    }
    for k, g in got.items():
        w = case["want"][k]
        assert g.shape == w.shape
        assert rel(g, w) < TOL[prec], (k, rel(g, w))
        assert site_max(g, w) < 10 * TOL[prec], (k, site_max(g, w))
    dd.close()


def test_one_slab_is_the_plain_operator(api, case):
    lat, psi = case["lat"], case["psi"]
    dd = api.Decomposition(case["L"], case["op"], 1)
    assert rel(dd.D(psi, "f64"), case["want"]["D"]) < TOL["f64"]
    assert rel(dd.Dhat(np.ascontiguousarray(psi[:, lat.even]), "f64"), case["want"]["Dhat"]) < TOL["f64"]
    dd.close()


@pytest.mark.parametrize("nparts", [2, 4])
def test_decomposed_solve_matches_oracle(api, case, nparts):
    lat, psi, eo = case["lat"], case["psi"], case["eo"]
    if lat.dims[3] % (2 * nparts):
        pytest.skip("slabs of an odd number of time slices")
    dd = api.Decomposition(case["L"], case["op"], nparts)
    x, info = dd.solve(psi, api.make_solver(tol=1e-11))
    for k in range(psi.shape[0]):
        assert info[k]["status"] == 0 and info[k]["true_rel_residual"] <= 1e-11, info[k]
        xe, _ = solvers.bicgstab(eo.schur, eo.prepare(psi[k]), tol=1e-14)
        want = eo.reconstruct(xe, psi[k])
        assert rel(x[k], want) < 1e-10, (k, rel(x[k], want))
        # the same FP64 recursion as the oracle's BiCGStab (the decomposed solve stops at
        # |r| <= 0.1 tol |b^|): a wrong step length still converges, but takes many more iterations
        _, ref = solvers.bicgstab(eo.schur, eo.prepare(psi[k]), tol=1e-12)
        assert abs(info[k]["inner_iters"] - ref["iters"]) <= max(3, ref["iters"] // 10), (info[k], ref)
    dd.close()


def test_plan_and_bad_arguments(api):
    from paper_2303_05883_gb300 import _abi

    p = api.bridge_dd_plan_of((4, 6, 4, 8), 4, 3)
    assert p["local_dims"] == (4, 6, 4, 2) and p["t0"] == 6 and p["rank_up"] == 0 and p["rank_down"] == 2
    assert p["up_wraps"] == 1 and p["down_wraps"] == 0 and p["face_sites"] == 48
    with pytest.raises(_abi.BridgeError):
        api.bridge_dd_plan_of((4, 6, 4, 8), 3, 0)  # Lt not divisible
    with pytest.raises(_abi.BridgeError):
        api.bridge_dd_plan_of((4, 6, 4, 8), 8, 0)  # slabs of one time slice
    L = api.Lattice((4, 4, 4, 8))
    with pytest.raises(_abi.BridgeError) as e:
        api.Decomposition(L, api.make_op("wilson", 0.12), 2)
    assert e.value.status == _abi.BRIDGE_ESTATE  # no gauge field yet
    L.close()
