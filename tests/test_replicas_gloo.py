"""bench.py's N > 1 path (replicas only: no collective on the data path) with
two gloo ranks on the CPU: the job time is the slowest rank's, and the job
throughput counts every rank's units."""
import os

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t = bench.max_over_ranks(1.0 + rank * 0.5, world, "cpu")
    rate = bench.job_rate(100.0, world, t)
    q.put((rank, t, rate))
    dist.destroy_process_group()


def test_two_replicas_max_time_and_job_rate():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    ps = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    assert [t for _, t, _ in res] == [1.5, 1.5]
    assert [r for _, _, r in res] == [200.0 / 1.5] * 2


def test_single_rank_passthrough():
    import bench
    assert bench.max_over_ranks(2.0, 1, "cpu") == 2.0
    assert bench.job_rate(10.0, 1, 2.0) == 5.0
