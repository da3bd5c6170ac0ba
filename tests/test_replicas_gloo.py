"""Replica path of bench.py (one process per GPU, no data-path collective) on
CPU with world size 2 over gloo: the job time is the slowest rank's, the
whole-job rate counts every rank's points, and each replica draws its own
inputs from the shared recipe."""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        ms = 10.0 + 5.0 * rank  # rank 1 is the slow one
        ms_max = bench.max_over_ranks(ms, world, torch.device("cpu"))
        rate = bench.whole_job_rate(1000, world, ms_max)
        pr = bench.replica_problem(rank, 64)
        q.put((rank, ms_max, rate, pr.src.copy()))
    finally:
        dist.destroy_process_group()


def test_replicas_max_time_and_own_inputs():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort(key=lambda r: r[0])
    for rank, ms_max, rate, _ in res:
        assert ms_max == 15.0
        assert rate == pytest.approx(2 * 1000 / 0.015 / 1e6)
    assert not np.array_equal(res[0][3], res[1][3])


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, 1, None) == 3.5
    assert bench.whole_job_rate(10 ** 6, 1, 1000.0) == pytest.approx(1.0)
