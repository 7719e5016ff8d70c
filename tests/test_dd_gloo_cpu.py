"""The face schedule of the domain decomposition on two gloo ranks (CPU).

Each rank takes the slab that the library's plan (bridge_dd_plan_of, host
arithmetic only) assigns to it, builds the two faces the plan describes --
(1 - gamma_t) psi of its first time slice for the slab below and
U_t^dagger (1 + gamma_t) psi of its last slice for the slab above, in face
site order -- sends them to the ranks the plan names, and forms the Wilson
operator on its slab from the oracle's hopping term with the t boundary
left open plus the received faces (with the plan's wrap phases).  The
result must equal the oracle's operator on the whole lattice at the slab's
sites, and the all-reduce of per-slab partial sums must equal the global
dot product: the exchange pattern, the face indexing, the phases and the
reduction are checked with real message passing, no GPU involved.
"""

import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

DIMS, KAPPA, BC = (4, 6, 4, 8), 0.12, (1, 1, 1, -1)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, q):
    import torch
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import synth
        from oracle import dirac
        from oracle.gamma import GAMMA
        from oracle.lattice import Lattice
        from paper_2303_05883_gb300 import api

        plan = api.bridge_dd_plan_of(DIMS, world, rank)
        U = synth.gauge_field(DIMS, 0.4, 3)
        psi = synth.gaussian_spinor(DIMS, 3)
        Vs = DIMS[0] * DIMS[1] * DIMS[2]
        lt = plan["local_dims"][3]
        lo = plan["canon_offset_sites"]
        Us = np.ascontiguousarray(U[:, lo:lo + lt * Vs])
        ps = np.ascontiguousarray(psi[lo:lo + lt * Vs])
        loc = Lattice(plan["local_dims"])
        I4 = np.eye(4, dtype=np.complex128)
        Pm, Pp = I4 - GAMMA[3], I4 + GAMMA[3]

        def face_order(t_slice):
            # lexicographic sites of one slice, per parity, in face-site order f = s // 2
            s = np.arange(Vs)
            out = {}
            for par in (0, 1):
                lex = t_slice * Vs + s
                sel = loc.parity[lex] == par
                out[par] = lex[sel]
                assert np.array_equal(s[sel] // 2, np.arange(plan["face_sites"]))
            return out

        first, last = face_order(0), face_order(lt - 1)
        # faces: per parity of the sending site
        up_face = {par: np.einsum("st,ntc->nsc", Pm, ps[first[par]]) for par in (0, 1)}
        dn_face = {par: np.einsum("nba,nsb->nsa", Us[3][last[par]].conj(), np.einsum("st,ntc->nsc", Pp, ps[last[par]]))
                   for par in (0, 1)}
        pack = lambda f: torch.from_numpy(np.stack([f[0], f[1]]).view(np.float64).copy())  # noqa: E731
        recv_up = torch.empty_like(pack(up_face))  # from rank_up: its first slice
        recv_dn = torch.empty_like(pack(dn_face))  # from rank_down: its last slice
        # tag 0: first-slice faces (travel down), tag 1: last-slice faces (travel up)
        ops = [dist.P2POp(dist.isend, pack(up_face), plan["rank_down"], tag=0),
               dist.P2POp(dist.isend, pack(dn_face), plan["rank_up"], tag=1),
               dist.P2POp(dist.irecv, recv_up, plan["rank_up"], tag=0),
               dist.P2POp(dist.irecv, recv_dn, plan["rank_down"], tag=1)]
        for w in dist.batch_isend_irecv(ops):
            w.wait()
        from_up = recv_up.numpy().view(np.complex128)
        from_dn = recv_dn.numpy().view(np.complex128)
        # interior: the oracle hop on the slab with the t boundary open
        bc_open = (BC[0], BC[1], BC[2], 0)
        H = dirac.hop(Us, ps, loc, bc_open)
        ph_up = BC[3] if plan["up_wraps"] else 1
        ph_dn = BC[3] if plan["down_wraps"] else 1
        for par in (0, 1):
            # forward t hop from the last slice: (1 - gamma_t) U_t(x) psi(x + t) = U_t(x) [face of the slab above],
            # the receiving site of parity par meets the sender's first-slice site of parity 1 - par
            xs = last[par]
            H[xs] += ph_up * np.einsum("nab,nsb->nsa", Us[3][xs], from_up[1 - par])
            # backward t hop from the first slice: the slab below sent U^dag (1 + gamma_t) psi
            xs = first[par]
            H[xs] += ph_dn * from_dn[1 - par]
        Dloc = ps - KAPPA * H
        want = dirac.wilson(U, psi, Lattice(DIMS), KAPPA, BC)[lo:lo + lt * Vs]
        err = float(np.linalg.norm(Dloc - want) / np.linalg.norm(want))
        # the scalar all-reduce of the solver: <psi, D psi> summed over slabs
        part = torch.tensor([np.vdot(ps, Dloc).real, np.vdot(ps, Dloc).imag], dtype=torch.float64)
        dist.all_reduce(part)
        full = np.vdot(psi, dirac.wilson(U, psi, Lattice(DIMS), KAPPA, BC))
        q.put((rank, err, abs(complex(part[0].item(), part[1].item()) - full) / abs(full)))
    finally:
        dist.barrier()
        dist.destroy_process_group()


def test_two_slab_face_schedule_and_all_reduce():
    pytest.importorskip("torch.distributed")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(300)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=5) for _ in range(2))
    assert [g[0] for g in got] == [0, 1]
    for rank, err, red in got:
        assert err < 1e-14, (rank, err)
        assert red < 1e-13, (rank, red)
