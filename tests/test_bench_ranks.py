"""bench.py's multi-GPU path is replicas: the job time is the slowest rank's, the work every rank's.

Checked with two gloo ranks on the CPU (127.0.0.1 rendezvous): each rank reports its own time
and work; both must see max time and the summed work.
"""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = 100.0 + 50.0 * rank           # rank 1 is slower
        units = 1.0e9 * (rank + 1)         # and did more work
        q.put((rank, bench.aggregate_ranks(ms, units, world)))
    finally:
        dist.destroy_process_group()


def test_replica_aggregation_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    out = dict(q.get(timeout=10) for _ in range(2))
    for r in (0, 1):
        max_ms, rate = out[r]
        assert max_ms == pytest.approx(150.0)
        assert rate == pytest.approx(3.0e9 / 0.150)


def test_single_rank_aggregation():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate_ranks(200.0, 4.0e9, 1) == (200.0, pytest.approx(2.0e10))
