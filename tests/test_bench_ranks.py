"""The multi-rank host logic of bench.py on CPU: two gloo ranks, each with
its own timing, agree on the slowest rank's time, and the job's rate counts
both replicas over that time."""
import os
import socket

import pytest


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist

    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = 10.0 + 5.0 * rank            # rank 1 is the slow one
        worst = bench.max_over_ranks(mine, world, "cpu")
        q.put((rank, worst, bench.job_rate(1000, 4, world, worst * 1e-3)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [g[1] for g in got] == [15.0, 15.0]
    # 2 ranks x 1000 rays x 4 steps in 15 ms
    assert got[0][2] == pytest.approx(2 * 1000 * 4 / 15e-3 / 1e6)


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.job_rate(16, 2, 1, 1e-6) == pytest.approx(32.0)
