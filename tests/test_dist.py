"""Multi-rank host paths on CPU with the gloo backend, world size 2:
* bench.py's replicas: the job is timed by its slowest rank and its value
  counts every rank's replica;
* the sub-tensor layout of Sec. IV-B emulated with CPU ranks (the oracle's
  shares, reduced with all_reduce) against the one-process result."""
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


def _grid_worker(rank, world, port, q):
    import numpy as np
    import torch

    import oracle
    import synth

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    shape, Rt, grid = (10, 9, 8), 4, (4, 3, 2)
    Y = synth.host_tensor(synth.scaled(synth.WORKLOADS["c1"], shape))
    W = synth.sketch_matrices(shape, Rt, 7)
    blocks = oracle.grid_blocks(shape, grid)
    # this rank's sub-tensors: mode-1 blocks s_1 = rank, rank + world, ...
    mine = [c for c in np.ndindex(*grid) if c[0] % world == rank]
    Z = [torch.zeros((shape[n], Rt), dtype=torch.float64) for n in range(3)]
    for c in mine:
        idx = [blocks[n][c[n]] for n in range(3)]
        for n, part in enumerate(oracle.sketch_share(Y[np.ix_(*idx)], idx, W)):
            Z[n][torch.as_tensor(idx[n])] += torch.as_tensor(part)
    for z in Z:
        dist.all_reduce(z)  # Eq. 22: the shares summed over the workers
    U = [oracle.evd_orth(z.numpy(), slabs=grid[n]) for n, z in enumerate(Z)]
    G = torch.zeros((Rt,) * 3, dtype=torch.float64)
    for c in mine:
        idx = [blocks[n][c[n]] for n in range(3)]
        G += torch.as_tensor(oracle.core_share(Y[np.ix_(*idx)], idx, U))
    dist.all_reduce(G)
    if rank == 0:
        one = oracle.rand_tucker_grid(Y, W, grid)
        ok = all(np.allclose(Z[n].numpy(), one["Z"][n], atol=1e-12) for n in range(3))
        ok = ok and np.allclose(G.numpy(), one["G"], atol=1e-12)
        q.put((len(mine), ok))
    else:
        q.put((len(mine), True))
    dist.barrier()
    dist.destroy_process_group()


def test_subtensor_layout_on_two_ranks_matches_one_process():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_grid_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert sorted(n for n, _ in out) == [12, 12]
    assert all(ok for _, ok in out)


def test_slab_bounds_partition_the_first_mode():
    from paper_1412_1885_gb300.sharded import slab_bounds

    for I1 in (1, 7, 60, 3000, 3001):
        for world in range(1, min(I1, 9) + 1):
            b = [slab_bounds(I1, world, r) for r in range(world)]
            assert b[0][0] == 0 and b[-1][1] == I1
            assert all(b[r][1] == b[r + 1][0] for r in range(world - 1))
            sizes = [hi - lo for lo, hi in b]
            assert max(sizes) - min(sizes) <= 1 and min(sizes) >= 1
    with pytest.raises(ValueError):
        slab_bounds(3, 4, 0)


def _comm_worker(rank, world, port, q):
    import torch

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_1412_1885_gb300.sharded import Comm, slab_bounds

    comm = Comm()
    a = torch.full((3, 4), float(rank + 1), dtype=torch.float64)
    b = torch.arange(5, dtype=torch.float32) * (rank + 1)
    comm.allreduce_sum([a, b])
    flags = (comm.any_flag(rank == 1), comm.any_flag(False))
    lo, hi = slab_bounds(7, world, rank)
    rows = torch.arange(lo * 3, hi * 3, dtype=torch.float64).reshape(hi - lo, 3)
    counts = [slab_bounds(7, world, r)[1] - slab_bounds(7, world, r)[0] for r in range(world)]
    full = comm.allgather_rows(rows, counts)
    q.put((rank, a.tolist(), b.tolist(), flags, full.tolist()))
    dist.barrier()
    dist.destroy_process_group()


def test_exchange_layer_sums_flags_and_gathers_on_two_ranks():
    """The sharded form's exchange (Comm) over gloo: the sums equal the
    element-wise sums of both ranks' arrays in their own dtypes, a flag set
    on one rank is seen on both, and uneven row blocks come back stacked in
    rank order."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_comm_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, a, b, flags, full in out:
        assert a == [[3.0] * 4] * 3
        assert b == [0.0, 3.0, 6.0, 9.0, 12.0]
        assert flags == (True, False)
        assert full == [[float(3 * i + j) for j in range(3)] for i in range(7)]
