"""GPU parity of the two multi-pass compressions: Alg. 2 as printed
(tucker_seq, Khatri-Rao test matrices) and RandTucker2i (Alg. 3,
tucker_refine), through the C ABI, against the FP64 oracle.

Each step is checked on its own: for mode n the oracle takes the factors the
GPU produced for the earlier steps, forms the same Z_n, and its Householder
basis is compared with the GPU's basis for that mode.  So an error is charged
to the step that made it instead of compounding over the modes.  The
tolerances come from the arithmetic of each form:
  * FP64 data (CUDA cores): every sum in FP64; two orthonormal bases of the
    same Z differ by about cond(Z) rounding units (helpers.basis_tol), with a
    factor 10 for the shrunk tensor being formed in a different order;
  * FP32 and BF16 data: the shrunk tensors are FP32 and the tensor-core
    passes split U (and FP32 data) into two BF16 terms, which keeps about 16
    significant bits: a relative error of a few 1e-6 in Z_n, so the bases
    differ by at most EPS32 * cond(Z_n) with EPS32 = 1e-4 (a factor >= 10
    over that).
The core is checked against the oracle's core of Y with the GPU's factors,
relative to the bound |Y| x_n |U_n|^T."""
import numpy as np
import pytest

import oracle
import synth
from helpers import basis_tol, core_abs_bound, dev_tensor, dev_W, host, recon_err, small_problem

pytestmark = pytest.mark.gpu

EPS32 = 1e-4


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


def _basis_check(U_gpu, Z, dtype, what):
    """U_gpu against the Householder basis of the oracle's Z (same sign
    convention: diag(R) > 0), and orthonormality."""
    Uo = oracle.householder_qr(Z)[0]
    cond = float(np.linalg.cond(Z))
    tol = 10 * basis_tol(Z) if dtype == "f64" else max(1e-6, EPS32 * cond)
    err = float(np.abs(U_gpu - Uo).max())
    assert err <= tol, (what, err, tol, cond)
    assert np.abs(U_gpu.T @ U_gpu - np.eye(U_gpu.shape[1])).max() < 1e-12, what


def _core_check(Y, U, G, dtype):
    ref = oracle.tucker_core(Y, U)
    bnd = core_abs_bound(Y, U)
    # FP32 sums, plus up to three hi + lo splits (each below 2^-17 of the
    # value) on the tensor-core passes
    tol = 1e-11 if dtype == "f64" else 2e-5 + 3 * 2.0 ** -17
    assert np.all(np.abs(G - ref) <= tol * bnd), float((np.abs(G - ref) / bnd).max())


SEQ_CASES = [
    ("f64", "simt", (67, 45, 130), (4, 5, 3), 3),
    ("f32", "simt", (67, 45, 130), (4, 5, 3), 3),
    ("bf16", "simt", (67, 45, 130), (4, 5, 3), 3),
    ("f32", "tc", (67, 45, 128), (4, 5, 3), 3),
    ("bf16", "tc", (300, 260, 136), (10, 12, 9), 6),   # ragged: 300 = 4 x 64 + 44 rows, 138.1 tiles of 256
    ("bf16", "tc", (12, 10, 9, 16), (3, 4, 2, 5), 2),  # 4-way, tensor-core shapes
    ("bf16", "tc", (9, 11, 7, 13), (2, 3, 2, 3), 2),   # no tensor-core shape: CUDA-core fallbacks
    ("f64", "simt", (30, 24), (5, 4), 2),              # N = 2
]


@pytest.mark.parametrize("dtype,prec,shape,ranks,p", SEQ_CASES)
def test_tucker_seq_matches_the_oracle_step_by_step(tdk, ctx, dtype, prec, shape, ranks, p):
    N = len(shape)
    Rt = [r + p for r in ranks]
    Y, W, _ = small_problem(shape, ranks, p, seed=61, dtype=dtype)
    U, G, nrm = tdk.tucker_seq(ctx, dev_tensor(Y, dtype), dev_W(W), ranks, p, prec)
    assert ctx.sync_status() == 0
    Uh = [host(u) for u in U]
    Om = oracle.seq_test_matrices(shape, W)
    X = np.asarray(Y, dtype=np.float64)
    for n in range(N):
        Z = oracle.unfold(X, n) @ Om[n]
        _basis_check(Uh[n], Z, dtype, ("mode", n))
        X = oracle.ttm(X, Uh[n], n)
    _core_check(Y, Uh, host(G), dtype)
    assert abs(float(nrm.item()) - oracle.norm2(Y)) <= 1e-6 * oracle.norm2(Y)
    # end to end: the oracle's own run from the same inputs
    ref = oracle.rand_tucker_seq_krp(Y, W)
    e_gpu, e_or = recon_err(float(nrm.item()), host(G)), recon_err(ref["normY2"], ref["G"])
    assert abs(e_gpu - e_or) <= (1e-9 if dtype == "f64" else 1e-4), (e_gpu, e_or)


def test_tucker_seq_with_seeded_matrices_matches_explicit_ones(tdk, ctx):
    """W = NULL draws the one-pass sketch's seeded matrices; the sequential
    form reads their leading rows, so passing the drawn matrices gives the
    same bits."""
    shape, ranks, p = (40, 36, 48), (4, 4, 4), 4
    Y, _, _ = small_problem(shape, ranks, p, seed=8, dtype="bf16")
    Yd = dev_tensor(Y, "bf16")
    U1, G1, n1 = tdk.tucker_seq(ctx, Yd, None, ranks, p, "tc", seed=1234)
    W = tdk.sketch_matrices(ctx, shape, ranks, p, 1234)
    U2, G2, n2 = tdk.tucker_seq(ctx, Yd, W, ranks, p, "tc")
    assert ctx.sync_status() == 0
    assert all(np.array_equal(host(a), host(b)) for a, b in zip(U1, U2))
    assert np.array_equal(host(G1), host(G2)) and float(n1.item()) == float(n2.item())


def test_sequential_form_is_more_accurate_than_one_pass(tdk, ctx):
    """Noisy tensor (SNR 10 dB): Alg. 2's sketch of the shrunk tensor fits
    better than the one-pass sketch at the same widths, on the GPU as in the
    oracle (reconstruction error ||Y - [[G; U]]|| / ||Y|| by Pythagoras)."""
    shape, ranks, p = (96, 80, 64), (6, 6, 6), 6
    Ys = synth.tucker_dense(shape, ranks, 3)
    Y = synth.to_storage(synth.add_noise(Ys, 10.0, 3), "bf16")
    W = synth.sketch_matrices(shape, [r + p for r in ranks], 3)
    Yd, Wd = dev_tensor(Y, "bf16"), dev_W(W)
    _, Gs, ns = tdk.tucker_seq(ctx, Yd, Wd, ranks, p, "tc")
    U1, _ = tdk.tucker_sketch(ctx, Yd, Wd, ranks, p, "tc")
    G1, n1 = tdk.tucker_core(ctx, Yd, U1, ranks, p, "tc")
    e_seq, e_one = recon_err(float(ns.item()), host(Gs)), recon_err(float(n1.item()), host(G1))
    assert e_seq < e_one, (e_seq, e_one)


REFINE_CASES = [
    ("f64", "simt", (40, 36, 32), (5, 6, 7)),
    ("f32", "simt", (40, 36, 32), (5, 6, 7)),
    ("f32", "tc", (40, 36, 32), (5, 6, 6)),
    ("bf16", "tc", (200, 150, 136), (8, 10, 6)),
    ("bf16", "tc", (14, 12, 10, 16), (3, 4, 3, 5)),
    ("bf16", "simt", (14, 12, 10, 16), (3, 4, 3, 5)),
]


@pytest.mark.parametrize("dtype,prec,shape,ranks", REFINE_CASES)
def test_refine_pass_matches_the_oracle_step_by_step(tdk, ctx, dtype, prec, shape, ranks):
    """One tucker_refine pass: mode n's X uses the GPU's refined factors for
    p < n and the pass's input factors for p > n (Alg. 3); each mode's basis
    against the oracle's basis of that Z_n.  Two passes, then the core."""
    p = 2
    N = len(shape)
    Rt = [r + p for r in ranks]
    Y, _, _ = small_problem(shape, ranks, p, seed=53, dtype=dtype)
    U = [dev_tensor(u, "f64") for u in synth.random_factors(shape, Rt, 53)]
    Yd = dev_tensor(Y, dtype)
    for it in range(2):
        Wp = synth.refine_matrices(Rt, 53, it)
        U_in = [host(u) for u in U]
        tdk.tucker_refine(ctx, Yd, dev_W(Wp), U, ranks, p, prec=prec)
        assert ctx.sync_status() == 0
        U_out = [host(u) for u in U]
        for n in range(N):
            X = np.asarray(Y, dtype=np.float64)
            for q in range(N):
                if q != n:
                    X = oracle.ttm(X, U_out[q] if q < n else U_in[q], q)
            Z = oracle.unfold(X, n) @ oracle.khatri_rao([Wp[n][k] for k in range(N) if k != n])
            _basis_check(U_out[n], Z, dtype, ("pass", it, "mode", n))
    G, nrm = tdk.tucker_core(ctx, Yd, U, ranks, p, prec)
    _core_check(Y, [host(u) for u in U], host(G), dtype)


@pytest.mark.parametrize("dtype,prec,shape", [
    ("bf16", "tc", (300, 260, 136)),    # 4 full 64-row chunks + 44 rows; 138.1 column tiles of 256
    ("bf16", "tc", (130, 8, 9, 16)),    # B = 1152: 4.5 tiles
    ("bf16", "simt", (67, 45, 130)),
    ("f32", "tc", (67, 45, 128)),       # FP32 data: CUDA cores
    ("f64", "simt", (31, 17, 11)),
])
def test_leading_mode_contraction_matches_oracle_elementwise(tdk, dtype, prec, shape):
    """X = Y x_1 U_1^T alone (the test library's hook), every entry against
    the oracle's TTM, relative to the bound |Y| x_1 |U_1|^T: FP32 sums plus
    the hi + lo split of U (below 2^-17) on the tensor cores."""
    import ctypes

    import torch

    c = tdk.Context(0, testing=True)
    try:
        Rt0 = 60 if shape[0] >= 60 else 7
        ranks, p = [Rt0 - 4] + [3] * (len(shape) - 1), 4
        Y, _, _ = small_problem(shape, ranks, p, seed=71, dtype=dtype)
        U1 = np.linalg.qr(np.random.default_rng(71).standard_normal((shape[0], Rt0)))[0]
        Yd, Ud = dev_tensor(Y, dtype), dev_tensor(U1, "f64")
        B = int(np.prod(shape[1:]))
        X = torch.empty((Rt0, B), dtype=torch.float64 if dtype == "f64" else torch.float32, device="cuda")
        desc = tdk.make_desc(shape, tdk._dtype_code(Yd), ranks, p, prec)
        c._bind_stream()
        rc = c.L.tdk_test_ttm_lead(c.handle, ctypes.byref(desc), ctypes.c_void_p(Yd.data_ptr()),
                                   ctypes.c_void_p(Ud.data_ptr()), ctypes.c_void_p(X.data_ptr()))
        assert rc == 0 and c.sync_status() == 0
        ref = oracle.ttm(Y, U1, 0).reshape(Rt0, B)
        bnd = oracle.ttm(np.abs(Y), np.abs(U1), 0).reshape(Rt0, B)
        tol = 1e-13 if dtype == "f64" else 2e-5 + 2.0 ** -17
        err = np.abs(host(X) - ref)
        assert np.all(err <= tol * bnd), float((err / bnd).max())
    finally:
        c.close()
