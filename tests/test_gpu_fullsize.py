"""The benchmark workloads at their full sizes, end to end through the public
API, against the FP64 oracle on the same tensor and the same test matrices:

  * 1000^3 FP32 (CP rank 10, correlated factors, SNR 20 dB; R_n = 10, p = 10,
    R = 10) in the tensor-core form and in the plain CUDA-core form;
  * 200^4 FP32 nonnegative (CP rank 20, U[0, 1] factors, SNR 25 dB, clipped;
    R_n = 20, p = 10, nonnegative R = 20).

The library draws the test matrices from the workload's seed; the oracle
draws the same ones with its own generator.  The oracle reads the device
tensor block by block and runs the sub-tensor form of Sec. IV-B (sketch
shares, then core shares, summed), which the CPU pins equate with the
one-block computation, so that the FP64 work fits in host memory.

Acceptance, as stated for the method: the relative reconstruction error of
the Tucker model differs from the oracle's by at most 1e-5 (FP32 data), and
the FFCP factors from the same start reach a congruence of at least 0.999
after permutation and scaling."""
import numpy as np
import pytest

import oracle
import synth
from helpers import host, recon_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tdk():
    import paper_1412_1885_gb300 as t
    from paper_1412_1885_gb300 import build

    build.build()
    return t


@pytest.fixture(scope="module")
def ctx(tdk):
    c = tdk.Context(0)
    yield c
    c.close()


def _oracle_tucker_by_blocks(Y, W, grid):
    """Oracle sketch, Householder bases and core of the device tensor Y from
    its sub-tensors (Eq. 19 grid), each copied to the host in FP64."""
    import torch

    shape = tuple(Y.shape)
    N = len(shape)
    blocks = oracle.grid_blocks(shape, grid)
    cells = list(np.ndindex(*grid))
    Rt = [W[n][(n + 1) % N].shape[1] for n in range(N)]
    Z = [np.zeros((shape[n], Rt[n])) for n in range(N)]

    def sub(idx):
        sl = tuple(slice(int(ix[0]), int(ix[-1]) + 1) for ix in idx)
        return Y[sl].to(torch.float64).cpu().numpy()

    normY2 = 0.0
    for cell in cells:
        idx = [blocks[n][cell[n]] for n in range(N)]
        Ys = sub(idx)
        normY2 += float(np.sum(Ys * Ys))
        for n, part in enumerate(oracle.sketch_share(Ys, idx, W)):
            Z[n][idx[n]] += part
    U = [oracle.householder_qr(z)[0] for z in Z]
    G = np.zeros(Rt)
    for cell in cells:
        idx = [blocks[n][cell[n]] for n in range(N)]
        G += oracle.core_share(sub(idx), idx, U)
    return {"Z": Z, "U": U, "G": G, "normY2": normY2}


@pytest.fixture(scope="module")
def c2(tdk):
    import torch

    w = synth.WORKLOADS["c2"]
    Y, _ = synth.device_tensor(w, device="cuda")
    seed = synth.omega_seed(w)
    Wo = oracle.philox.sketch_matrices(seed, w.shape, w.Rt)
    ref = _oracle_tucker_by_blocks(Y, Wo, (20, 1, 1))
    B0 = synth.init_factors(w.Rt, w.als_R, w.seed)
    o = oracle.cp_als(ref["G"], B0, max_sweeps=w.als_max_sweeps, tol=w.als_tol)
    yield w, Y, seed, ref, B0, o
    del Y
    torch.cuda.empty_cache()


@pytest.mark.parametrize("prec", ["tc", "simt"])
def test_1000_cubed_fp32_end_to_end_matches_oracle(tdk, ctx, c2, prec):
    import torch

    w, Y, seed, ref, B0, o = c2
    out = tdk.decompose(ctx, Y, None, w.ranks, w.p, w.als_R, prec, max_sweeps=w.als_max_sweeps, tol=w.als_tol,
                        B0=[torch.as_tensor(b, device="cuda") for b in B0], seed=seed)
    assert ctx.sync_status() == 0
    e_gpu = recon_err(float(out["normY2"].item()), host(out["G"]))
    e_or = recon_err(ref["normY2"], ref["G"])
    print(f"{prec}: reconstruction error {e_gpu:.9f} (oracle {e_or:.9f}); sweeps {out['sweeps']} "
          f"(oracle {o['sweeps']}); fit_core {out['fit_core']:.9f} (oracle {o['fit']:.9f})")
    assert abs(e_gpu - e_or) <= 1e-5, (e_gpu, e_or)
    for n in range(3):
        Un = host(out["U"][n])
        assert np.abs(Un.T @ Un - np.eye(Un.shape[1])).max() < 1e-12
    Ao = oracle.lift(ref["U"], o["B"], o["lam"])
    cong = oracle.congruence(Ao, [host(a) for a in out["A"]])
    assert cong >= 0.999, cong
    assert abs(out["fit_core"] - o["fit"]) <= 1e-4


def test_200_pow4_fp32_nonneg_end_to_end_matches_oracle(tdk, ctx):
    import torch

    w = synth.WORKLOADS["c3"]
    Y, _ = synth.device_tensor(w, device="cuda")
    seed = synth.omega_seed(w)
    try:
        A0 = synth.init_factors(w.shape, w.als_R, w.seed, dist="uniform")
        out = tdk.decompose(ctx, Y, None, w.ranks, w.p, w.als_R, "tc", nonneg=True, max_sweeps=w.als_max_sweeps,
                            tol=w.als_tol, A0=[torch.as_tensor(a, device="cuda") for a in A0], seed=seed)
        assert ctx.sync_status() == 0
        Wo = oracle.philox.sketch_matrices(seed, w.shape, w.Rt)
        ref = _oracle_tucker_by_blocks(Y, Wo, (10, 10, 1, 1))
    finally:
        del Y
        torch.cuda.empty_cache()
    e_gpu = recon_err(float(out["normY2"].item()), host(out["G"]))
    e_or = recon_err(ref["normY2"], ref["G"])
    o = oracle.cp_als_nonneg(ref["G"], ref["U"], A0, max_sweeps=w.als_max_sweeps, tol=w.als_tol)
    print(f"reconstruction error {e_gpu:.9f} (oracle {e_or:.9f}); sweeps {out['sweeps']} (oracle {o['sweeps']}); "
          f"fit_core {out['fit_core']:.9f} (oracle {o['fit']:.9f})")
    assert abs(e_gpu - e_or) <= 1e-5, (e_gpu, e_or)
    Ah = [host(a) for a in out["A"]]
    assert all(np.all(a >= 0) for a in Ah)
    Ao = [a.copy() for a in o["A"]]
    Ao[-1] = Ao[-1] * o["lam"][None, :]
    cong = oracle.congruence(Ao, Ah)
    assert cong >= 0.999, cong
