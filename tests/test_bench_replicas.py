"""bench.py with N > 1: independent replicas, one per rank (the path has no
exchange step).  The whole-job rate is the units of all ranks over the slowest
rank's time; checked here with two gloo ranks on the CPU."""
import os
import socket
import sys

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sys.path.insert(0, ROOT)
    import bench
    # rank r processed (r + 1) * 1e12 units in 10 * (r + 1) ms
    rate, slow = bench.replica_rate((rank + 1) * 1e12, 10.0 * (rank + 1), dist, "cpu")
    q.put((rank, rate, slow))
    dist.barrier()
    dist.destroy_process_group()


def test_replica_rate_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # (1 + 2) * 1e12 units over the slower rank's 20 ms, identical on both ranks
    for rank, rate, slow in out:
        assert slow == pytest.approx(20.0)
        assert rate == pytest.approx(3e12 / 20e-3)


def test_replica_rate_single_process():
    sys.path.insert(0, ROOT)
    import bench
    rate, slow = bench.replica_rate(5e12, 50.0)
    assert slow == 50.0 and rate == pytest.approx(1e14)
