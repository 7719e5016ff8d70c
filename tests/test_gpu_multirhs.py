"""Multi-RHS stencils against the FP64 oracle, element by element.

Twelve right-hand sides on one gauge field (the paper's O(10) equations per
configuration, Sec. 3) go through the stencil kernels with a pinned launch
shape: the per-thread kernel (variant 0), the shared-link tile kernel with
and without a register cap (variants 9, 10: the eight links and T^-1 of a
site staged once in shared memory for all right-hand sides of a 32-site
tile), the same with the neighbour spinors of the next hop copied into
shared memory while the current hop computes (variants 11, 12; 16-bit
storage, FP32 falls back to variant 0), and the 2-4
right-hand-sides-per-thread kernels (6-8).  The lattice
has a ragged last tile (720 sites per parity = 22.5 tiles) and several site
blocks; 13 right-hand sides make two tile groups (7 + 6) with one idle warp.
Each comparison bounds the relative L2 error over the whole output and the
largest per-site error against the RMS site norm, so that an error confined
to a face or a tail cannot hide in the L2 sum.
"""

import numpy as np
import pytest

import synth
from oracle import evenodd, solvers
from oracle.lattice import Lattice

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-13, "f32": 2e-6, "f16": 5e-3, "bf16": 5e-3}
PREC_ID = {"f64": 0, "f32": 1, "f16": 2, "bf16": 3}
DIMS = (6, 6, 4, 10)
KAPPA, CSW = 0.125, 1.0


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def site_max(a, b):
    """Largest per-site error over the RMS per-site norm of b."""
    e = np.linalg.norm((a - b).reshape(a.shape[0], a.shape[1], -1), axis=2)
    n = np.linalg.norm(b.reshape(b.shape[0], b.shape[1], -1), axis=2)
    return float(e.max() / np.sqrt(np.mean(n ** 2)))


def check(got, want, prec, what=""):
    assert got.shape == want.shape
    e, m = rel(got, want), site_max(got, want)
    assert e < TOL[prec], f"{what} {prec}: rel L2 {e:.3e}"
    assert m < 10 * TOL[prec], f"{what} {prec}: per-site max {m:.3e}"


@pytest.fixture(scope="module")
def api():
    import __graft_entry__ as g

    g.build()
    from paper_2303_05883_gb300 import api

    return api


@pytest.fixture(scope="module")
def mr(api):
    lat = Lattice(DIMS)
    U = synth.gauge_field(DIMS, 0.3, 41)
    psi = synth.gaussian_spinor(DIMS, 41, nrhs=13)
    eo = evenodd.EvenOdd(U, lat, KAPPA, CSW)
    op = api.make_op("clover", KAPPA, CSW)
    L = api.Lattice(DIMS)
    L.upload(U, op)
    want = {
        "Deo": np.stack([eo.D_hop(0, p[lat.odd]) for p in psi]),
        "Doe": np.stack([eo.D_hop(1, p[lat.even]) for p in psi]),
        "Dhat": np.stack([eo.schur(p[lat.even]) for p in psi]),
    }
    yield dict(lat=lat, U=U, psi=psi, eo=eo, op=op, L=L, want=want)
    L.close()


def pin(api, L, prec, flags, red, nrhs, variant, nblk=3):
    key = "x".join(map(str, DIMS))
    api.bridge_tune_set(L.handle, f"hop/{PREC_ID[prec]}/{flags}/{red}/{key}/{nrhs}", 64, nblk, variant)


@pytest.mark.parametrize("nrhs", [12, 13])
@pytest.mark.parametrize("variant", [0, 9, 10, 11, 12, 8])
@pytest.mark.parametrize("prec", ["f32", "f16", "bf16"])
def test_deo_and_schur_multi_rhs(api, mr, prec, variant, nrhs):
    lat, L, op = mr["lat"], mr["L"], mr["op"]
    psi = mr["psi"][:nrhs]
    pin(api, L, prec, 0, 0, nrhs, variant)  # D_eo / D_oe
    pin(api, L, prec, 4, 0, nrhs, variant)  # Schur pass 1 (T^-1 epilogue)
    check(L.Deo(op, np.ascontiguousarray(psi[:, lat.odd]), 0, prec), mr["want"]["Deo"][:nrhs], prec, "D_eo")
    check(L.Deo(op, np.ascontiguousarray(psi[:, lat.even]), 1, prec), mr["want"]["Doe"][:nrhs], prec, "D_oe")
    check(L.Dhat(op, np.ascontiguousarray(psi[:, lat.even]), prec), mr["want"]["Dhat"][:nrhs], prec, "D^")


@pytest.mark.parametrize("prec,variant", [("f32", 9), ("f16", 11), ("f16", 12)])
@pytest.mark.parametrize("nblk", [1, 2, 7, 1000])
def test_tile_kernel_grid_sizes(api, mr, nblk, prec, variant):
    """One block looping over every tile, a few, and more blocks than tiles."""
    lat, L, op = mr["lat"], mr["L"], mr["op"]
    psi = mr["psi"][:12]
    pin(api, L, prec, 0, 0, 12, variant, nblk=nblk)
    check(L.Deo(op, np.ascontiguousarray(psi[:, lat.odd]), 0, prec), mr["want"]["Deo"][:12], prec, "D_eo")


@pytest.mark.parametrize("variant", [0, 9, 10, 11])
@pytest.mark.parametrize("prec", ["f32", "f16", "bf16"])
def test_twelve_rhs_solve_with_pinned_kernels(api, mr, prec, variant):
    """A 12-RHS mixed solve whose Schur passes (with their fused <rhat, v> and
    (<t, s>, |t|^2) reductions) and D_eo run on the pinned kernel, against
    the oracle's even-odd BiCGStab solution of each system."""
    lat, L, op, eo = mr["lat"], mr["L"], mr["op"], mr["eo"]
    B = mr["psi"][:12]
    for flags, red in [(0, 0), (4, 0), (5, 2), (5, 3)]:
        pin(api, L, prec, flags, red, 12, variant)
    X, info = L.solve(op, B, api.make_solver(tol=1e-12, inner_prec=prec))
    if "x" not in mr:
        xs = []
        for k in range(12):
            xe, _ = solvers.bicgstab(eo.schur, eo.prepare(B[k]), tol=1e-14)
            xs.append(eo.reconstruct(xe, B[k]))
        mr["x"] = np.stack(xs)
    for k in range(12):
        assert info[k]["status"] == 0, (k, info[k])
        assert rel(X[k], mr["x"][k]) < 1e-10, (k, rel(X[k], mr["x"][k]))


@pytest.mark.parametrize("variant", [9, 11])
def test_tile_kernel_repeat_is_bit_identical(api, mr, variant):
    """The tile kernel's fused reductions sum in a fixed order."""
    lat, L, op = mr["lat"], mr["L"], mr["op"]
    B = mr["psi"][:12]
    for flags, red in [(0, 0), (4, 0), (5, 2), (5, 3)]:
        pin(api, L, "f16", flags, red, 12, variant)
    s = api.make_solver(tol=1e-11, inner_prec="f16")
    a, _ = L.solve(op, B, s)
    b, _ = L.solve(op, B, s)
    assert np.array_equal(a, b)
