"""One worker of the sharded-form GPU test (run by torch.distributed.run with
the gloo backend; several workers may share one GPU because no kernel waits
on another worker: the exchange runs on the host).  Writes this worker's
results to OUT_rank.npz.

    sharded_worker.py OUT DTYPE PREC SEEDED
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, HERE)
sys.path.insert(0, os.path.dirname(HERE))

import numpy as np  # noqa: E402
import torch  # noqa: E402
import torch.distributed as dist  # noqa: E402

import synth  # noqa: E402
from helpers import dev_tensor, dev_W, small_problem  # noqa: E402

SHAPE, RANKS, P, R, SEED = (61, 40, 64), (5, 4, 6), 3, 4, 4242


def main():
    out, dtype, prec, seeded = sys.argv[1], sys.argv[2], sys.argv[3], sys.argv[4] == "1"
    dist.init_process_group("gloo")
    import paper_1412_1885_gb300 as t
    from paper_1412_1885_gb300.sharded import Comm, decompose_sharded, slab_bounds

    comm = Comm()
    torch.cuda.set_device(0)
    Y, W, _ = small_problem(SHAPE, RANKS, P, seed=31, dtype=dtype, R_cp=R)
    lo, hi = slab_bounds(SHAPE[0], comm.world, comm.rank)
    Ys = dev_tensor(Y[lo:hi], dtype)
    ctx = t.Context(0)
    B0 = [torch.as_tensor(b, device="cuda") for b in synth.init_factors([r + P for r in RANKS], R, 5)]
    o = decompose_sharded(ctx, comm, Ys, lo, SHAPE[0], RANKS, P, R, prec, W=None if seeded else dev_W(W),
                          seed=SEED, max_sweeps=40, tol=0.0, B0=B0)
    assert ctx.sync_status() == 0
    np.savez(f"{out}_{comm.rank}.npz", G=o["G"].double().cpu().numpy(), normY2=float(o["normY2"].item()),
             U=np.concatenate([u.cpu().numpy().ravel() for u in o["U"]]),
             A=np.concatenate([a.cpu().numpy().ravel() for a in o["A"]]), fit=o["fit_core"], sweeps=o["sweeps"],
             lo=lo, hi=hi)
    ctx.close()
    dist.barrier()
    dist.destroy_process_group()


if __name__ == "__main__":
    main()
