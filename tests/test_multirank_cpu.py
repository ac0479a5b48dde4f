"""The benchmark's multi-rank host logic on CPU ranks (gloo, world size 2):
each rank refines its own workload replica, and the whole-job value uses the
slowest rank's time and the sum of the ranks' units."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms, units = bench.aggregate_ranks(10.0 + 5.0 * rank, 1000 + rank, dist, "cpu")
    q.put((rank, ms, units))
    dist.destroy_process_group()


def test_aggregate_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, ms, units in res:
        assert ms == 15.0 and units == 2001


def test_single_rank_passthrough():
    import bench
    assert bench.aggregate_ranks(3.5, 7, None, "cpu") == (3.5, 7)
