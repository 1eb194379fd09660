"""Sharded form of the method over several workers (Sec. IV-B).

Y is split along its first mode into slabs of consecutive rows, one per
worker (a one-dimensional case of the sub-tensor grid of Eq. 19).  Every
arithmetic step runs in libtdk's kernels on the worker's own GPU; between
the steps the workers sum small arrays, which is the whole exchange:

  1. sketch shares (tucker_sketch_partial): the rows of Z_1 are the slab's
     own; the Z_n of the other modes are summed over the workers (Eq. 22);
  2. U_n, n >= 2, from the summed Z_n on every worker (same bits in, same
     bits out);
  3. U_1 by CholQR2 over the row blocks of Z_1: the Gram of the stacked
     blocks is the sum of the blocks' Grams (Eq. 23, with a Cholesky factor
     in place of the eigendecomposition), two rounds.  If a Cholesky pivot
     breaks down on any worker (a numerically rank-deficient Z_1), the
     workers gather Z_1 and complete its basis as the one-GPU path does;
  4. core shares (tucker_core_partial) with the slab's rows of U_1, summed
     with the shares of ||Y||^2;
  5. FFCP on the summed core, on every worker, with U_1 gathered for the
     lift (I_1 x (R_1 + p) values).

`Comm` is the exchange: sums and row gathers over a torch.distributed
process group.  With NCCL the buffers stay on the GPU; with gloo (CPU tests,
or several processes sharing one GPU) they go through host memory.  The
exchanged arrays are FP64: the sums are exact up to the order of addition,
and every worker receives the same result.
"""
from __future__ import annotations

from . import (TDK_WRANKDEF, Context, ffcp_als, gram, orth, orth_apply, tucker_core_partial,
               tucker_sketch_partial, _dtype_code)


def slab_bounds(I1: int, world: int, rank: int):
    """Rows [lo, hi) of mode 1 owned by `rank`: near-equal contiguous slabs,
    the first I1 mod world slabs one row longer."""
    if not (0 <= rank < world) or I1 < world:
        raise ValueError("every worker needs at least one row")
    base, extra = divmod(int(I1), int(world))
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


class Comm:
    """Sums and row gathers over a torch.distributed process group (the
    default group when `group` is None)."""

    def __init__(self, group=None):
        import torch.distributed as dist

        self.dist = dist
        self.group = group
        self.world = dist.get_world_size(group)
        self.rank = dist.get_rank(group)
        self.on_device = dist.get_backend(group) == "nccl"

    def allreduce_sum(self, tensors):
        """Sum every tensor over the workers, in place.  One flat FP64 buffer
        carries them all (one collective per exchange step)."""
        import torch

        if self.world == 1 or not tensors:
            return tensors
        dev = tensors[0].device if self.on_device else torch.device("cpu")
        flat = torch.cat([t.reshape(-1).to(device=dev, dtype=torch.float64) for t in tensors])
        self.dist.all_reduce(flat, op=self.dist.ReduceOp.SUM, group=self.group)
        o = 0
        for t in tensors:
            n = t.numel()
            t.copy_(flat[o:o + n].reshape(t.shape).to(device=t.device, dtype=t.dtype))
            o += n
        return tensors

    def any_flag(self, flag: bool) -> bool:
        """True on every worker if `flag` is set on any worker."""
        import torch

        if self.world == 1:
            return bool(flag)
        t = torch.tensor([1.0 if flag else 0.0], dtype=torch.float64)
        if self.on_device:
            t = t.cuda()
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX, group=self.group)
        return bool(t.item() > 0.0)

    def allgather_rows(self, t, counts):
        """Stack every worker's row block (rows counts[r] on worker r) in
        worker order; every worker receives the whole matrix."""
        import torch

        if self.world == 1:
            return t
        dev = t.device if self.on_device else torch.device("cpu")
        width = max(counts)
        buf = torch.zeros((width,) + tuple(t.shape[1:]), dtype=t.dtype, device=dev)
        buf[:t.shape[0]] = t.to(dev)
        parts = [torch.empty_like(buf) for _ in range(self.world)]
        self.dist.all_gather(parts, buf, group=self.group)
        return torch.cat([p[:c] for p, c in zip(parts, counts)]).to(t.device)


def rand_tucker_sharded(ctx: Context, comm: Comm, Y_slab, row_off: int, I1: int, ranks, p, prec="tc", W=None,
                        seed=0):
    """Steps 1-4 on this worker's slab Y_slab (rows [row_off, row_off +
    Y_slab.shape[0]) of mode 1 of a tensor with I1 rows).  W: the whole
    tensor's test matrices, or None to draw them from `seed` on every worker.
    Returns dict(U1_rows, U (U[0] the slab's rows of U_1), G, normY2, counts,
    rankdef)."""
    import torch

    N = Y_slab.dim()
    counts = [slab_bounds(I1, comm.world, r)[1] - slab_bounds(I1, comm.world, r)[0] for r in range(comm.world)]
    if counts[comm.rank] != Y_slab.shape[0] or slab_bounds(I1, comm.world, comm.rank)[0] != row_off:
        raise ValueError("the slab does not match slab_bounds for this worker")
    Z = tucker_sketch_partial(ctx, Y_slab, row_off, I1, W, ranks, p, prec, seed)
    comm.allreduce_sum(Z[1:])
    U = [None] + [orth(ctx, Z[n]) for n in range(1, N)]
    rankdef = bool(ctx.sync_status() & TDK_WRANKDEF)
    U1 = Z[0]
    broke = False
    for _round in range(2):
        g = gram(ctx, U1)
        comm.allreduce_sum([g])
        U1 = orth_apply(ctx, g, U1)
        # every worker factors the same Gram, so a breakdown shows on all of them
        broke = comm.any_flag(bool(ctx.sync_status() & TDK_WRANKDEF))
        if broke:
            break
    if broke:
        # a rank-deficient Z_1: gather it and complete the basis as tucker_sketch does
        Z1 = comm.allgather_rows(Z[0], counts)
        U1 = orth(ctx, Z1)[row_off:row_off + counts[comm.rank]].contiguous()
        ctx.sync_status()
        rankdef = True
    U[0] = U1
    G, nrm = tucker_core_partial(ctx, Y_slab, I1, U, ranks, p, prec)
    nrm = nrm.reshape(1)
    comm.allreduce_sum([G, nrm])
    torch.cuda.current_stream().synchronize()
    return {"U": U, "G": G, "normY2": nrm.reshape(()), "counts": counts, "rankdef": rankdef}


def decompose_sharded(ctx: Context, comm: Comm, Y_slab, row_off: int, I1: int, ranks, p, R, prec="tc", W=None,
                      seed=0, **als):
    """The whole path on the workers: rand_tucker_sharded, then FFCP on the
    summed core on every worker with U_1 gathered (step 5).  `als` takes the
    keyword arguments of ffcp_als (max_sweeps, tol, nonneg, init, B0, A0...).
    Returns ffcp_als's dict with U (full), G and normY2 added."""
    tk = rand_tucker_sharded(ctx, comm, Y_slab, row_off, I1, ranks, p, prec, W, seed)
    U = list(tk["U"])
    U[0] = comm.allgather_rows(U[0], tk["counts"])
    shape = (int(I1),) + tuple(Y_slab.shape[1:])
    if als.get("init", "given") == "given" and als.get("B0") is None and als.get("A0") is None:
        als["init"] = "hosvd"
    out = ffcp_als(ctx, tk["G"], U, shape, ranks, p, _dtype_code(Y_slab), R, normY2=tk["normY2"], **als)
    out.update({"U": U, "G": tk["G"], "normY2": tk["normY2"], "rankdef": tk["rankdef"]})
    return out
