"""The continuous-batching request engine on the GPU.

A request's result must be the same alone and in a mix of concurrently
running requests (stated tolerance 1e-10; the engine uses deterministic
reductions and fixed launch shapes, so the mix is expected bit-identical),
and must match the FP64 oracle.  Admission respects the memory budget and
the slot limit; requests larger than the whole budget are refused.
"""

import time

import numpy as np
import pytest

import synth
from oracle import evenodd, solvers
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


@pytest.fixture(scope="module")
def lattices(api):
    out = {}
    for dims, eps, seed in [((4, 4, 4, 8), 0.2, 11), ((8, 8, 8, 8), 0.3, 12), ((4, 6, 8, 10), 0.25, 13)]:
        L = api.Lattice(dims)
        U = synth.gauge_field(dims, eps, seed)
        L.upload(U)
        out[dims] = (L, U)
    yield out
    for L, _ in out.values():
        L.close()


def _mix(api, lattices):
    reqs = []
    rng = np.random.default_rng(0)
    for i, dims in enumerate(list(lattices) * 3):
        kind = "clover" if i % 2 else "wilson"
        op = api.make_op(kind, float(rng.uniform(0.11, 0.125)), 1.0 if kind == "clover" else 0.0)
        nrhs = int(rng.integers(1, 4))
        b = synth.gaussian_spinor(dims, 50 + i, nrhs=nrhs)
        prec = ["f32", "f16", "bf16"][i % 3]
        reqs.append((dims, op, b, api.make_solver(tol=1e-11, inner_prec=prec)))
    return reqs


def test_alone_equals_in_mix(api, lattices):
    reqs = _mix(api, lattices)
    alone = []
    for dims, op, b, s in reqs:
        h = api.bridge_submit(lattices[dims][0].handle, op, s, b)
        st, x, info = api.bridge_wait(h)
        api.bridge_request_release(h)
        assert st == 0
        alone.append(x)
    # all at once: the engine overlaps them on the GPU
    hs = [api.bridge_submit(lattices[dims][0].handle, op, s, b) for dims, op, b, s in reqs]
    spans = []
    for (dims, op, b, s), h, xa in zip(reqs, hs, alone):
        st, x, info = api.bridge_wait(h)
        _, t_admit, t_done = api.bridge_request_times(h)
        spans.append((t_admit, t_done))
        api.bridge_request_release(h)
        assert st == 0 and all(i["true_rel_residual"] <= 1e-11 for i in info)
        assert rel(x, xa) <= 1e-10
        assert np.array_equal(x, xa)  # deterministic reductions: identical bits
    # the mix really ran concurrently: some requests were on the GPU together
    overlaps = sum(1 for i in range(len(spans)) for j in range(i + 1, len(spans))
                   if spans[i][0] < spans[j][1] and spans[j][0] < spans[i][1])
    assert overlaps >= 1, spans


def test_engine_results_match_oracle(api, lattices):
    dims = (4, 6, 8, 10)
    L, U = lattices[dims]
    kappa, csw = 0.12, 1.0
    op = api.make_op("clover", kappa, csw)
    b = synth.gaussian_spinor(dims, 77, nrhs=2)
    h = api.bridge_submit(L.handle, op, api.make_solver(tol=1e-12), b)
    st, x, info = api.bridge_wait(h)
    api.bridge_request_release(h)
    assert st == 0
    eo = evenodd.EvenOdd(U, Lattice(dims), kappa, csw)
    for k in range(2):
        xe, _ = solvers.bicgstab(eo.schur, eo.prepare(b[k]), tol=1e-14)
        assert rel(x[k], eo.reconstruct(xe, b[k])) < 1e-10


def test_poll_pending_then_done_and_times_ordered(api, lattices):
    L, _ = lattices[(8, 8, 8, 8)]
    op = api.make_op("wilson", 0.12)
    b = synth.gaussian_spinor((8, 8, 8, 8), 3, nrhs=4)
    h = api.bridge_submit(L.handle, op, api.make_solver(tol=1e-12, check_every=1, use_graph=0), b)
    r = api.bridge_poll(h)
    # it may already be done on a fast GPU; either way the final poll returns OK
    deadline = time.time() + 60
    while r is None and time.time() < deadline:
        time.sleep(0.001)
        r = api.bridge_poll(h)
    assert r is not None and r[0] == 0
    ts, ta, td = api.bridge_request_times(h)
    assert ts <= ta <= td
    api.bridge_request_release(h)


def test_request_over_budget_is_refused(api, lattices):
    from paper_2303_05883_gb300 import _abi

    api.bridge_engine_config(budget_bytes=1 << 20)  # 1 MiB: nothing fits
    try:
        L, _ = lattices[(8, 8, 8, 8)]
        with pytest.raises(_abi.BridgeError) as e:
            api.bridge_submit(L.handle, api.make_op("wilson", 0.12), api.make_solver(), synth.gaussian_spinor((8, 8, 8, 8), 1))
        assert e.value.status == _abi.BRIDGE_ENOMEM
    finally:
        api.bridge_engine_config(budget_bytes=64 << 30)


def test_one_slot_admits_in_fifo_order(api, lattices):
    """With one slot, equal requests are admitted one at a time, in arrival order."""
    L, _ = lattices[(4, 4, 4, 8)]
    op = api.make_op("wilson", 0.12)
    api.bridge_engine_config(budget_bytes=64 << 30, max_active=1)
    try:
        bs = [synth.gaussian_spinor((4, 4, 4, 8), 200 + i) for i in range(4)]
        hs = [api.bridge_submit(L.handle, op, api.make_solver(tol=1e-10), b) for b in bs]
        times = []
        for h in hs:
            st, x, info = api.bridge_wait(h, timeout_ms=60000)
            assert st == 0
            times.append(api.bridge_request_times(h))
            api.bridge_request_release(h)
        for (s0, a0, d0), (s1, a1, d1) in zip(times, times[1:]):
            assert s0 <= s1 and a0 <= a1 and d0 <= d1
    finally:
        api.bridge_engine_config(budget_bytes=64 << 30, max_active=16)


def test_wait_timeout_and_release_of_running_request(api, lattices):
    L, _ = lattices[(8, 8, 8, 8)]
    op = api.make_op("wilson", 0.1249)  # near critical: many iterations
    b = synth.gaussian_spinor((8, 8, 8, 8), 9, nrhs=12)
    h = api.bridge_submit(L.handle, op, api.make_solver(tol=1e-14, max_iter=200000, inner_prec="f16"), b)
    r = api.bridge_wait(h, timeout_ms=0)
    if r is None:  # still running: release cancels it
        api.bridge_request_release(h)
    else:
        api.bridge_request_release(h)
    # the engine keeps serving afterwards
    h2 = api.bridge_submit(L.handle, api.make_op("wilson", 0.1), api.make_solver(tol=1e-10), synth.gaussian_spinor((8, 8, 8, 8), 10))
    st, x, info = api.bridge_wait(h2, timeout_ms=60000)
    api.bridge_request_release(h2)
    assert st == 0


def test_borrowed_rhs_equals_copied_and_release_while_queued(api, lattices):
    """A borrowed b (read in place at admission) gives the bit-identical result
    of a copied one.  Borrowed requests released at once -- queued ones
    withdrawn, admitted ones cancelled after their upload -- leave the engine
    serving, and their arrays can then be freed."""
    L, _ = lattices[(8, 8, 8, 8)]
    op = api.make_op("clover", 0.12, 1.0)
    s = api.make_solver(tol=1e-10)
    b = synth.gaussian_spinor((8, 8, 8, 8), 31, nrhs=3)
    h1 = api.bridge_submit(L.handle, op, s, b)
    h2 = api.bridge_submit(L.handle, op, s, b.copy(), borrow=True)
    st1, x1, _ = api.bridge_wait(h1, timeout_ms=60000)
    st2, x2, _ = api.bridge_wait(h2, timeout_ms=60000)
    api.bridge_request_release(h1)
    api.bridge_request_release(h2)
    assert st1 == 0 and st2 == 0 and np.array_equal(x1, x2)
    api.bridge_engine_config(budget_bytes=64 << 30, max_active=2)
    try:
        hs = [api.bridge_submit(L.handle, op, s, synth.gaussian_spinor((8, 8, 8, 8), 40 + i, nrhs=2), borrow=True)
              for i in range(12)]
        for h in hs:
            api.bridge_request_release(h)
        del hs
        h = api.bridge_submit(L.handle, op, s, b, borrow=True)
        st, x, _ = api.bridge_wait(h, timeout_ms=60000)
        api.bridge_request_release(h)
        assert st == 0 and np.array_equal(x, x1)
    finally:
        api.bridge_engine_config(budget_bytes=64 << 30, max_active=16)


def test_gauge_reupload_refused_while_requests_run(api):
    from paper_2303_05883_gb300 import _abi

    dims = (8, 8, 8, 8)
    L = api.Lattice(dims)
    U = synth.gauge_field(dims, 0.2, 4)
    L.upload(U)
    b = synth.gaussian_spinor(dims, 5, nrhs=12)
    h = api.bridge_submit(L.handle, api.make_op("wilson", 0.124), api.make_solver(tol=1e-13, inner_prec="f16"), b)
    # a submitted request holds the lattice from submission on, queued or running
    with pytest.raises(_abi.BridgeError) as e:
        L.upload(U)
    assert e.value.status == _abi.BRIDGE_ESTATE
    with pytest.raises(_abi.BridgeError) as e:
        api.bridge_lattice_destroy(L.handle)
    assert e.value.status == _abi.BRIDGE_ESTATE
    st, x, info = api.bridge_wait(h)
    assert st == 0
    L.upload(U)  # done requests no longer hold it
    api.bridge_request_release(h)
    L.close()


def test_release_of_queued_request_frees_the_lattice(api):
    dims = (8, 8, 8, 8)
    api.bridge_engine_config(max_active=1)
    try:
        L = api.Lattice(dims)
        U = synth.gauge_field(dims, 0.2, 6)
        L.upload(U)
        op = api.make_op("wilson", 0.1249)
        slv = api.make_solver(tol=1e-12, inner_prec="f32")
        b = synth.gaussian_spinor(dims, 7, nrhs=12)
        h1 = api.bridge_submit(L.handle, op, slv, b)
        h2 = api.bridge_submit(L.handle, op, slv, b)  # queued behind the long-running h1
        api.bridge_request_release(h2)
        api.bridge_wait(h1)
        api.bridge_request_release(h1)
        L.upload(U)  # nothing holds the lattice now
        L.close()
    finally:
        api.bridge_engine_config(max_active=64)
