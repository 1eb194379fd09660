"""Shared helpers for the GPU parity tests (inputs from `synth`, expected
values from `oracle`; nothing here computes the method)."""
import numpy as np

import oracle
import synth

TORCH_DT = {"f64": "float64", "f32": "float32", "bf16": "bfloat16"}
DT_CODE = {"f64": 0, "f32": 1, "bf16": 2}


# element-wise sketch tolerance of the CUDA-core form, relative to the bound
# sum |y| * prod |w| of each entry (FP64: rounding of FP64 FMAs; FP32
# accumulation for F32 and BF16 data)
TOL_SKETCH = {("f64", "simt"): 1e-12, ("f32", "simt"): 2e-5, ("bf16", "simt"): 2e-5}


def dev_tensor(Y: np.ndarray, dtype: str, device="cuda"):
    import torch

    t = torch.as_tensor(np.ascontiguousarray(Y), dtype=torch.float64)
    return t.to(getattr(torch, TORCH_DT[dtype])).to(device).contiguous()


def dev_W(W, device="cuda"):
    """Device copies of the sketch matrices; an array shared between modes
    (synth.sketch_matrices(shared=True)) stays one tensor."""
    return synth.device_sketch(W, device)


def host(t) -> np.ndarray:
    return t.detach().double().cpu().numpy()


def sketch_abs_bound(Y, W):
    """Elementwise |Y|_(n) |Omega_n|: the scale against which the rounding
    error of a computed sketch entry is bounded (|sum a_i b_i| <= sum |a_i||b_i|)."""
    Z, _ = oracle.sketch(np.abs(Y), [[None if w is None else np.abs(w) for w in row] for row in W])
    return Z


def core_abs_bound(Y, U):
    return oracle.tucker_core(np.abs(Y), [np.abs(u) for u in U])


def basis_tol(Z) -> float:
    """Distance to expect between two FP64 orthonormal bases of the same Z
    (CholQR2 against Householder, both with diag(R) > 0): the QR factors of Z
    move by about cond(Z) units of rounding; 1000 units of 2^-52 per unit of
    condition, and never below 1e-12."""
    return max(1e-12, 1e3 * 2.220446049250313e-16 * float(np.linalg.cond(np.asarray(Z, dtype=np.float64))))


def bf16_ulp(x) -> np.ndarray:
    """Spacing of the BF16 values (8 significant bits) at |x|: 2^(e - 7) for
    |x| in [2^e, 2^(e+1)), between 2^-8 and 2^-7 of |x|."""
    x = np.abs(np.asarray(x, dtype=np.float64))
    _, e = np.frexp(np.where(x > 0, x, 1.0))
    return np.where(x > 0, np.ldexp(1.0, e - 8), 0.0)


def recon_err(normY2: float, G: np.ndarray) -> float:
    """||Y - [[G; U]]|| / ||Y|| for orthonormal U (Pythagoras)."""
    return float(np.sqrt(max(0.0, normY2 - float(np.sum(np.asarray(G, dtype=np.float64) ** 2))) / normY2))


def small_problem(shape, ranks, p, seed, dtype="f32", snr=20.0, R_cp=None, dist="normal", clip0=False,
                  shared=False):
    R_cp = R_cp or min(ranks)
    A = synth.cp_factors(shape, R_cp, seed, dist)
    Y = synth.add_noise(synth.cp_dense(A), snr, seed, clip0)
    Y = synth.to_storage(Y, dtype)
    W = synth.sketch_matrices(shape, [r + p for r in ranks], seed, shared=shared)
    return Y, W, A
