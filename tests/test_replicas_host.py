"""The multi-rank path of bench.py (replicas only: every rank advances its
own independent problems, no data-path collective) on two gloo ranks on the
CPU: the timed region is the slowest rank's, every rank agrees on it, the
whole-job value counts every rank's particles, and ranks draw different
problems (their seeds differ)."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, _ = bench.dist_env()
        local_ms = 10.0 + 5.0 * rank                      # rank 1 is the slower one
        total = bench.max_over_ranks(local_ms, dist)
        value = bench.replica_throughput(1000, w, 4, total)
        import numpy as np
        from paper_1009_2768_gb300 import synth
        first = float(synth.rng(r).random())              # the replica's seed is its rank
        q.put((r, w, total, value, first))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time_and_sum_the_particles():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    assert [o[0] for o in out] == [0, 1] and all(o[1] == 2 for o in out)
    assert all(o[2] == 15.0 for o in out)                 # max over ranks, on every rank
    assert all(abs(o[3] - 1000 * 2 * 4 / 0.015) < 1e-6 for o in out)
    assert out[0][4] != out[1][4]                         # independent replicas


def test_single_process_needs_no_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(12.5) == 12.5
    assert bench.replica_throughput(10, 1, 5, 1000.0) == 50.0
