"""The multi-rank host path of bench.py (independent replicas, one per rank)
on CPU with the gloo backend, world size 2: the job is timed by its slowest
rank and its value counts every rank's replica."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    ms = bench.max_over_ranks(10.0 + 5.0 * rank, dist, "cpu")
    value = bench.job_value(4_000_000_000, world, ms)
    q.put((rank, ms, value))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_replicas_are_timed_by_the_slowest_rank(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    slowest = 10.0 + 5.0 * (world - 1)
    for rank, ms, value in out:
        assert ms == slowest
        assert abs(value - world * 4.0 / (slowest * 1e-3)) < 1e-9


def test_single_process_needs_no_group():
    import bench

    assert bench.max_over_ranks(3.5, None, "cpu") == 3.5
    assert abs(bench.job_value(8_000_000_000, 1, 1000.0) - 8.0) < 1e-12
