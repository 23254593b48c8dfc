"""Multi-GPU runs are replicas: each rank solves its own system with no
collective on the data path, and bench.py reports the whole job's updates over
the slowest rank's time.  The host-side aggregation runs here as two gloo
ranks on the CPU."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        updates, seconds = bench.job_totals(dist, "cpu", 1000 * (rank + 1), 0.5 + rank)
        out.put((rank, updates, seconds))
    finally:
        dist.destroy_process_group()


def test_replica_totals_over_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    for rank, updates, seconds in got:
        assert updates == pytest.approx(3000.0)  # 1000 + 2000
        assert seconds == pytest.approx(1.5)     # the slowest rank


def test_single_process_totals_pass_through():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.job_totals(None, "cpu", 123, 0.25) == (123.0, 0.25)
