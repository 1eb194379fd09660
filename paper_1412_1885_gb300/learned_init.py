"""Training set, training loop and evaluation of the learned FFCP
initialiser (the tdk_mlp part of the C ABI).  Every step runs in libtdk.so;
this module only sequences the calls and keeps the device arrays.

A training sample is produced by the method itself: a tensor is compressed
(tucker_sketch, tucker_core), FFCP runs on its core to convergence, and the
sample keeps the core, the column sums of its Tucker factors (for the
canonical sign rule), the rank R and the converged factors with the weights
absorbed (G ~ [[B*]]).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import F64, MLP_PARAMS, Context, Mlp, _dtype_code, ffcp_als, tucker_core, tucker_sketch


@dataclass
class Samples:
    G: object        # FP32 device [n, Rt^N]
    colsums: object  # FP64 device [n, N, Rt]
    R: object        # int32 device [n]
    Bstar: object    # FP64 device [n, N, Rt, Rt], normalised columns
    lam: object      # FP64 device [n, Rt], their weights
    sweeps: list     # ALS sweeps the method needed from its own start
    fit: list        # converged core fit


def method_sample(ctx: Context, model: Mlp, Y, W, ranks, p, R, B0, prec="tc", max_sweeps=1000, tol=1e-7,
                  init="given", seed=0):
    """Compress Y (W = None: test matrices drawn from `seed`), run FFCP from
    B0 on its core; returns a dict with the flat FP32 core G, colsums
    [N, Rt], Bstar [N, Rt, Rt], R, sweeps, fit, U and the core in its own
    type (Gc) with ||Y||^2."""
    import torch

    N = Y.dim()
    Rt = int(ranks[0]) + int(p)
    nrm = torch.empty((), dtype=torch.float64, device=Y.device)
    U, _ = tucker_sketch(ctx, Y, W, ranks, p, prec, seed=seed, normY2=nrm)
    G, _ = tucker_core(ctx, Y, U, ranks, p, prec, want_norm=False)
    init = "given" if init in ("given", "rand") else init
    out = ffcp_als(ctx, G, U, tuple(Y.shape), ranks, p, _dtype_code(Y), R, max_sweeps, tol, init=init, B0=B0,
                   normY2=nrm)
    # zero-padded copies (columns >= R unused)
    Bs = torch.zeros((N, Rt, Rt), dtype=torch.float64, device=Y.device)
    lam = torch.zeros(Rt, dtype=torch.float64, device=Y.device)
    for n in range(N):
        Bs[n, :, :R].copy_(out["B"][n])
    lam[:R].copy_(out["lam"])
    cs = model.colsums(U, tuple(Y.shape), ranks, p)
    if _dtype_code(Y) == F64:
        raise ValueError("the learned initialiser trains on FP32 cores")
    # a run that stopped at max_sweeps, or whose weights dwarf the data (a
    # degenerate solution whose components cancel), is not a usable target
    lam_h = out["lam"].abs().max().item()
    nrm_h = float(nrm.item()) ** 0.5
    usable = out["sweeps"] < max_sweeps and lam_h <= 5.0 * nrm_h
    return {"G": G.reshape(-1), "colsums": cs, "Bstar": Bs, "lam": lam, "R": int(R), "sweeps": out["sweeps"],
            "fit": out["fit_core"], "U": U, "Gc": G, "normY2": nrm, "usable": usable}


def stack(items) -> Samples:
    """Samples from the usable method_sample results (converged, not
    degenerate)."""
    import torch

    items = [it for it in items if it["usable"]]
    G = torch.stack([it["G"] for it in items])
    cs = torch.stack([it["colsums"] for it in items])
    Bs = torch.stack([it["Bstar"] for it in items])
    lam = torch.stack([it["lam"] for it in items])
    R = torch.tensor([it["R"] for it in items], dtype=torch.int32, device=G.device)
    return Samples(G, cs, R, Bs, lam, [it["sweeps"] for it in items], [it["fit"] for it in items])


def train(model: Mlp, data: Samples, epochs: int, batch: int, lr: float = 1e-3, alpha: float = 0.5,
          seed: int = 0, lr_final: float | None = None, warmup: float = 0.05, clip: float = 1.0):
    """Adam over shuffled mini-batches; the step size rises linearly over the
    first `warmup` fraction of the steps, then decays linearly to lr_final
    (default lr / 10); every step's gradient is clipped to a global norm of
    `clip` (0: no clipping).  The parameters of the epoch with the lowest
    mean loss are kept.  Returns the mean loss of every epoch."""
    import torch

    n = int(data.G.shape[0])
    rng = np.random.default_rng(seed)
    steps = epochs * max(1, n // batch)
    lr_final = lr / 10 if lr_final is None else lr_final
    hist, k = [], 0
    best, best_params = None, None
    for _ in range(epochs):
        perm = torch.as_tensor(rng.permutation(n), device=data.G.device)
        tot, cnt = 0.0, 0
        for s in range(0, n - batch + 1, batch):
            idx = perm[s:s + batch]
            nw = max(1, int(warmup * steps))
            if k < nw:
                step_lr = lr * (k + 1) / nw
            else:
                step_lr = lr + (lr_final - lr) * (k - nw) / max(1, steps - nw - 1)
            tot += model.train_step(data.G[idx].contiguous(), data.colsums[idx].contiguous(), data.R[idx].contiguous(),
                                    data.Bstar[idx].contiguous(), alpha=alpha, lr=step_lr,
                                    lam=data.lam[idx].contiguous(), clip=clip)
            cnt += 1
            k += 1
        hist.append(tot / max(cnt, 1))
        if np.isfinite(hist[-1]) and (best is None or hist[-1] < best):
            best, best_params = hist[-1], model.get(MLP_PARAMS)
    if best_params is not None:
        model.set_params(best_params)
    return hist
