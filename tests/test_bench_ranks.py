"""The benchmark's multi-rank aggregation (replicas: one matrix per rank),
run as two gloo ranks on the CPU: every rank reports the slowest rank's
time, and the job rate counts the units of all ranks over that time."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

from tests.conftest import ROOT


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, out):
    import sys
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        local_ms = [120.0, 80.0][rank]
        t = bench.slowest(local_ms, ws)
        rate = bench.job_rate(6, ws, t / 1e3)
        out.put((rank, t, rate))
    finally:
        dist.destroy_process_group()


def test_two_rank_aggregation():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, rate in res:
        assert t == 120.0                      # the slowest rank's time on every rank
        assert abs(rate - 2 * 6 / 0.120) < 1e-9   # all ranks' SVDs over that time


def test_single_rank_is_local():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.slowest(42.0, 1) == 42.0
    assert bench.job_rate(10, 1, 2.0) == 5.0
