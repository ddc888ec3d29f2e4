"""The multi-GPU form of the benchmark is replicas only: every rank sorts its own
copy of the workload on its own GPU, with no collective on the data path; the
job's time is the slowest rank's and its work the sum over ranks.  The host-side
aggregation runs here as two gloo ranks on the CPU."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        ms, units = bench.aggregate(dist, ms=1.5 + rank, units=1000 * (rank + 1), device="cpu")
        q.put((rank, ms, units))
    finally:
        dist.destroy_process_group()


def test_two_replicas_max_time_sum_work():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, units in res:
        assert ms == pytest.approx(2.5)   # slowest rank
        assert units == 3000              # work of both ranks


def test_single_process_passthrough():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate(None, 3.25, 77, "cpu") == (3.25, 77)
