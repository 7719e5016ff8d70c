"""The N > 1 path of bench.py on CPU: two gloo ranks.

The solver path has no exchange step on one GPU, so N GPUs run N
independent replicas; the only cross-rank logic is the whole-job
aggregation (slowest rank's time, summed work), tested here with the gloo
backend and world size 2.
"""

import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, q):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    ms, nbytes = bench.aggregate_ranks(10.0 + 5.0 * rank, 1e9 * (rank + 1), device="cpu")
    q.put((rank, ms, nbytes))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_aggregation_takes_max_time_and_sums_work():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=5) for _ in range(2))
    for rank, ms, nbytes in got:
        assert ms == pytest.approx(15.0) and nbytes == pytest.approx(3e9)


def test_single_process_passthrough():
    import bench

    assert bench.aggregate_ranks(3.0, 7.0) == (3.0, 7.0)
