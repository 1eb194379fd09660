"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on the
same seeded inputs.  Sizes span several tiles with ragged tails; tolerances
are derived from the arithmetic of each form and stated per test."""
import math

import numpy as np
import pytest

import oracle
import synth
from helpers import (DT_CODE, TOL_SKETCH, core_abs_bound, dev_tensor, dev_W, host, recon_err, sketch_abs_bound,
                     small_problem)

pytestmark = pytest.mark.gpu

# TOL_SKETCH (helpers): relative rounding unit of the accumulation per form,
# times a safety factor: FP64: products and sums in FP64; FP32/BF16 data on
# CUDA cores: FP32 sums of up to ~1e6 terms (errors grow like sqrt(terms) * u32
# in practice).

SHAPES = [
    (67, 45, 130),        # 3015 rows (47 tiles of 64 + tail), 130 columns (4 chunks of 32 + tail)
    (9, 11, 7, 13),       # 4-way, tiny ragged
    (33, 70, 64),
]


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


@pytest.mark.parametrize("dtype,prec", [("f64", "simt"), ("f32", "simt"), ("bf16", "simt")])
@pytest.mark.parametrize("shape", SHAPES)
def test_sketch_matches_oracle(tdk, ctx, shape, dtype, prec):
    ranks = [min(4, s - 3) for s in shape]
    p = 3
    Y, W, _ = small_problem(shape, ranks, p, seed=11, dtype=dtype)
    U, Z = tdk.tucker_sketch(ctx, dev_tensor(Y, dtype), dev_W(W), ranks, p, prec, want_Z=True)
    Zo, _ = oracle.sketch(Y, W)
    bnd = sketch_abs_bound(Y, W)
    tol = TOL_SKETCH[(dtype, prec)]
    for n in range(len(shape)):
        err = np.abs(host(Z[n]) - Zo[n])
        assert np.all(err <= tol * bnd[n] + 1e-300), (n, float((err / bnd[n]).max()))
        Un = host(U[n])
        assert np.abs(Un.T @ Un - np.eye(Un.shape[1])).max() < 1e-12


def test_cholqr2_matches_householder_fp64(tdk, ctx):
    shape, ranks, p = (61, 47, 53), (5, 6, 7), 4
    Y, W, _ = small_problem(shape, ranks, p, seed=3, dtype="f64")
    U, _ = tdk.tucker_sketch(ctx, dev_tensor(Y, "f64"), dev_W(W), ranks, p, "simt")
    ref = oracle.rand_tucker(Y, W)
    for n in range(3):
        # same convention (positive diagonal of R) => same Q entrywise
        assert np.abs(host(U[n]) - ref["U"][n]).max() < 1e-10
    assert ctx.sync_status() == 0


def test_rank_deficient_sketch_is_completed(tdk, ctx):
    """Noise-free tensor of exact multilinear rank with p > 0: Z_n has rank R_n
    < R_n + p, Cholesky breaks down, the completion keeps U orthonormal and
    the Tucker reconstruction exact."""
    shape, ranks, p = (40, 36, 30), (3, 4, 5), 4
    Y = synth.tucker_dense(shape, ranks, 5)
    W = synth.sketch_matrices(shape, [r + p for r in ranks], 1)
    Yd = dev_tensor(Y, "f64")
    U, _ = tdk.tucker_sketch(ctx, Yd, dev_W(W), ranks, p, "simt")
    flags = ctx.sync_status()
    assert flags & tdk.TDK_WRANKDEF
    for u in U:
        un = host(u)
        assert np.abs(un.T @ un - np.eye(un.shape[1])).max() < 1e-12
    G, nrm = tdk.tucker_core(ctx, Yd, U, ranks, p, "simt")
    Yh = oracle.tucker_full(host(G), [host(u) for u in U])
    assert np.linalg.norm(Y - Yh) / np.linalg.norm(Y) < 1e-10


@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16"])
@pytest.mark.parametrize("shape", SHAPES)
def test_core_matches_oracle(tdk, ctx, shape, dtype):
    ranks = [min(4, s - 3) for s in shape]
    p = 3
    Y, W, _ = small_problem(shape, ranks, p, seed=5, dtype=dtype)
    ref = oracle.rand_tucker(Y, W)
    Ud = [dev_tensor(u, "f64") for u in ref["U"]]   # oracle U as input to the GPU core
    G, nrm = tdk.tucker_core(ctx, dev_tensor(Y, dtype), Ud, ranks, p, "simt")
    bnd = core_abs_bound(Y, ref["U"])
    tol = 1e-12 if dtype == "f64" else 2e-5
    err = np.abs(host(G) - ref["G"])
    assert np.all(err <= tol * bnd), float((err / bnd).max())
    assert math.isclose(float(nrm.item()), ref["normY2"], rel_tol=1e-12 if dtype == "f64" else 1e-6)


@pytest.mark.parametrize("prec,dtype", [("simt", "f32"), ("tc", "f32"), ("tc", "bf16"), ("simt", "f64")])
def test_core_wide_ranks_matches_oracle(tdk, ctx, prec, dtype):
    # sketch widths above 32 (the shrunk contractions take their wide-tile
    # form for FP32 cores): 3-way with ragged 64-tiles in every mode, and a
    # 4-way case whose middle contractions see Bd = 40 * 36 and 40 * 36 * 34
    for shape, ranks, p in [((70, 66, 72), (36, 40, 38), 2), ((38, 44, 40, 48), (34, 33, 36, 38), 2)]:
        Y, W, _ = small_problem(shape, ranks, p, seed=23, dtype=dtype)
        U = [np.linalg.qr(np.random.default_rng(24 + n).standard_normal((I, r + p)))[0]
             for n, (I, r) in enumerate(zip(shape, ranks))]
        Gref = oracle.tucker_core(Y, U)
        G, nrm = tdk.tucker_core(ctx, dev_tensor(Y, dtype), [dev_tensor(u, "f64") for u in U], ranks, p, prec)
        assert ctx.sync_status() == 0
        bnd = core_abs_bound(Y, U)
        tol = 1e-12 if dtype == "f64" else 2e-5 + (_tc_core_split(dtype) if prec == "tc" else 0.0)
        err = np.abs(host(G) - Gref)
        assert np.all(err <= tol * bnd), (shape, float((err / bnd).max()))


@pytest.mark.parametrize("prec,dtype", [("simt", "f64"), ("simt", "f32"), ("tc", "f32")])
@pytest.mark.parametrize("shape,ranks", [((600, 40, 64), (10, 12, 14)), ((300, 72, 64), (40, 36, 44)),
                                         ((520, 9, 10, 16), (6, 5, 7, 8))])
def test_core_split_contraction_matches_oracle(tdk, ctx, prec, dtype, shape, ranks):
    # a first mode of several hundred: the last contraction of the chain (one
    # output slab) is split over that mode and the partials summed in order
    p = 2
    Y, W, _ = small_problem(shape, ranks, p, seed=31, dtype=dtype)
    U = [np.linalg.qr(np.random.default_rng(32 + n).standard_normal((I, r + p)))[0]
         for n, (I, r) in enumerate(zip(shape, ranks))]
    Gref = oracle.tucker_core(Y, U)
    G, nrm = tdk.tucker_core(ctx, dev_tensor(Y, dtype), [dev_tensor(u, "f64") for u in U], ranks, p, prec)
    assert ctx.sync_status() == 0
    bnd = core_abs_bound(Y, U)
    tol = 1e-12 if dtype == "f64" else 2e-5 + (_tc_core_split(dtype) if prec == "tc" else 0.0)
    err = np.abs(host(G) - Gref)
    assert np.all(err <= tol * bnd), (shape, float((err / bnd).max()))


@pytest.fixture(params=["persistent", "multi"])
def als_form(request, ctx):
    ctx.set_als_form(request.param == "multi")
    yield request.param
    ctx.set_als_form(False)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_als_matches_oracle_on_same_core(tdk, ctx, dtype, als_form):
    shape, ranks, p, R = (50, 45, 40), (6, 6, 6), 4, 5
    Y, W, A = small_problem(shape, ranks, p, seed=9, dtype=dtype, snr=25.0, R_cp=R)
    ref = oracle.rand_tucker(Y, W)
    Rt = [r + p for r in ranks]
    B0 = synth.init_factors(Rt, R, 4)
    ref_als = oracle.cp_als(ref["G"], B0, max_sweeps=60, tol=0.0)
    Gd = dev_tensor(ref["G"], "f64" if dtype == "f64" else "f32")
    Ud = [dev_tensor(u, "f64") for u in ref["U"]]
    out = tdk.ffcp_als(ctx, Gd, Ud, shape, ranks, p, DT_CODE[dtype], R, max_sweeps=60, tol=0.0,
                       B0=[dev_tensor(b, "f64") for b in B0], check_every=16)
    assert out["sweeps"] == 60
    tol = 1e-10 if dtype == "f64" else 1e-5
    assert abs(out["fit_core"] - ref_als["fit"]) < tol
    Ah = [host(a) for a in out["A"]]
    Ao = oracle.lift(ref["U"], ref_als["B"], ref_als["lam"])
    assert oracle.congruence(Ao, Ah) > (1 - 1e-9 if dtype == "f64" else 0.9999)
    if dtype == "f64":
        for n in range(3):
            assert np.allclose(host(out["B"][n]), ref_als["B"][n], atol=1e-8)


def test_als_stopping_rule_matches_oracle_fp64(tdk, ctx, als_form):
    shape, ranks, p, R = (30, 28, 26), (4, 4, 4), 3, 3
    Y, W, _ = small_problem(shape, ranks, p, seed=2, dtype="f64", snr=30.0, R_cp=R)
    ref = oracle.rand_tucker(Y, W)
    B0 = synth.init_factors([r + p for r in ranks], R, 8)
    o = oracle.cp_als(ref["G"], B0, max_sweeps=500, tol=1e-9)
    out = tdk.ffcp_als(ctx, dev_tensor(ref["G"], "f64"), [dev_tensor(u, "f64") for u in ref["U"]], shape, ranks,
                       p, 0, R, max_sweeps=500, tol=1e-9, B0=[dev_tensor(b, "f64") for b in B0], check_every=4)
    assert out["sweeps"] == o["sweeps"]
    assert abs(out["fit_core"] - o["fit"]) < 1e-12


def test_nonneg_als_matches_oracle(tdk, ctx, als_form):
    shape, ranks, p, R = (24, 22, 20, 18), (5, 5, 5, 5), 3, 4
    Y, W, A = small_problem(shape, ranks, p, seed=7, dtype="f64", snr=25.0, R_cp=R, dist="uniform", clip0=True)
    ref = oracle.rand_tucker(Y, W)
    A0 = synth.init_factors(shape, R, 6, dist="uniform")
    o = oracle.cp_als_nonneg(ref["G"], ref["U"], A0, max_sweeps=40, tol=0.0)
    out = tdk.ffcp_als(ctx, dev_tensor(ref["G"], "f64"), [dev_tensor(u, "f64") for u in ref["U"]], shape, ranks,
                       p, 0, R, max_sweeps=40, tol=0.0, nonneg=True, A0=[dev_tensor(a, "f64") for a in A0])
    assert abs(out["fit_core"] - o["fit"]) < 1e-10
    Ah = [host(a) for a in out["A"]]
    assert all(np.all(a >= 0) for a in Ah)
    Ao = [a.copy() for a in o["A"]]
    Ao[-1] = Ao[-1] * o["lam"][None, :]
    for n in range(4):
        assert np.allclose(Ah[n], Ao[n], atol=1e-8)


def test_als_hosvd_start_matches_oracle(tdk, ctx, als_form):
    # HOSVD start (leading R left singular vectors of every G_(n), largest
    # entry positive), then 60 sweeps, FP64
    shape, ranks, p, R = (40, 36, 32), (5, 5, 5), 3, 4
    Y, W, _ = small_problem(shape, ranks, p, seed=12, dtype="f64", snr=25.0, R_cp=R)
    ref = oracle.rand_tucker(Y, W)
    o = oracle.cp_als(ref["G"], oracle.hosvd_init(ref["G"], R), max_sweeps=60, tol=0.0)
    out = tdk.ffcp_als(ctx, dev_tensor(ref["G"], "f64"), [dev_tensor(u, "f64") for u in ref["U"]], shape, ranks,
                       p, 0, R, max_sweeps=60, tol=0.0, init="hosvd")
    assert out["sweeps"] == 60
    assert abs(out["fit_core"] - o["fit"]) < 1e-10
    for n in range(3):
        assert np.allclose(host(out["B"][n]), o["B"][n], atol=1e-8)


def test_nonneg_als_hosvd_start_matches_oracle(tdk, ctx, als_form):
    # nonnegative form from |U_n B_n^hosvd|
    shape, ranks, p, R = (24, 22, 20), (5, 5, 5), 3, 4
    Y, W, _ = small_problem(shape, ranks, p, seed=13, dtype="f64", snr=25.0, R_cp=R, dist="uniform", clip0=True)
    ref = oracle.rand_tucker(Y, W)
    A0 = [np.abs(u @ b) for u, b in zip(ref["U"], oracle.hosvd_init(ref["G"], R))]
    o = oracle.cp_als_nonneg(ref["G"], ref["U"], A0, max_sweeps=30, tol=0.0)
    out = tdk.ffcp_als(ctx, dev_tensor(ref["G"], "f64"), [dev_tensor(u, "f64") for u in ref["U"]], shape, ranks,
                       p, 0, R, max_sweeps=30, tol=0.0, nonneg=True, init="hosvd")
    assert abs(out["fit_core"] - o["fit"]) < 1e-10


def test_end_to_end_c1_fp64(tdk, ctx):
    """Workload 1 at full size (100^3 FP64, CP rank 5, SNR 30 dB, p = 5, ALS
    rank 5, <= 100 sweeps, relative fit change < 1e-9)."""
    w = synth.WORKLOADS["c1"]
    Y = synth.host_tensor(w)
    W = synth.sketch_matrices(w.shape, w.Rt, w.seed)
    B0 = synth.init_factors(w.Rt, w.als_R, w.seed)
    ref = oracle.rand_tucker(Y, W)
    o = oracle.cp_als(ref["G"], B0, max_sweeps=w.als_max_sweeps, tol=w.als_tol)
    out = tdk.decompose(ctx, dev_tensor(Y, "f64"), dev_W(W), w.ranks, w.p, w.als_R, "simt",
                        max_sweeps=w.als_max_sweeps, tol=w.als_tol, B0=[dev_tensor(b, "f64") for b in B0])
    e_gpu = recon_err(float(out["normY2"].item()), host(out["G"]))
    e_or = recon_err(ref["normY2"], ref["G"])
    assert abs(e_gpu - e_or) < 1e-12
    assert abs(out["fit_core"] - o["fit"]) < 1e-10
    Ao = oracle.lift(ref["U"], o["B"], o["lam"])
    assert oracle.congruence(Ao, [host(a) for a in out["A"]]) > 0.999999
    # and the planted factors are found
    A_true = synth.cp_factors(w.shape, w.R_cp, w.seed)
    assert oracle.congruence(A_true, [host(a) for a in out["A"]]) > 0.99


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_end_to_end_scaled_fp32(tdk, ctx, dtype):
    """Workload 2's data model at 120^3: reconstruction-error difference <= 1e-5."""
    w = synth.scaled(synth.WORKLOADS["c2"], (120, 120, 120))
    w.dtype = dtype
    Y = synth.host_tensor(w)
    W = synth.sketch_matrices(w.shape, w.Rt, w.seed)
    ref = oracle.rand_tucker(Y, W)
    U, _ = tdk.tucker_sketch(ctx, dev_tensor(Y, dtype), dev_W(W), w.ranks, w.p, "simt")
    G, nrm = tdk.tucker_core(ctx, dev_tensor(Y, dtype), U, w.ranks, w.p, "simt")
    e_gpu = recon_err(float(nrm.item()), host(G))
    e_or = recon_err(ref["normY2"], ref["G"])
    assert abs(e_gpu - e_or) <= 1e-5, (e_gpu, e_or)


# ---------------------------------------------------------------- tensor-core form
# Shapes for the tcgen05 path: the contiguous mode times the element size is a
# multiple of 16 bytes (TMA row pitch).  They span ragged j-tiles (128 rows),
# ragged column ranges (256) and several p values.
TC_SHAPES = [
    (67, 45, 136),
    (9, 11, 7, 16),
    (5, 200, 264),
    (3, 130, 512),
]
# rounding of one BF16 operand (RNE): 2^-9 relative; FP32 data split hi+lo and
# KRP rows split hi+lo (sketch width <= 32): residual below 2^-17; KRP rows of
# a last mode wider than 32 are rounded once (2^-9), for either data type.
U_BF16 = 2.0 ** -9


def _tc_tol(dtype, mode_is_last, Rt_last):
    acc = 2e-5  # FP32 accumulation, as for the CUDA-core form
    if dtype == "bf16":
        return acc + (U_BF16 if mode_is_last else 0.0)
    # FP32 data: hi + lo everywhere, except the KRP rows of the last mode when
    # its sketch width exceeds 32 (no room for their lo half): one BF16 rounding
    return acc + (U_BF16 if (mode_is_last and Rt_last > 32) else 2.0 ** -16)


@pytest.mark.parametrize("dtype", ["bf16", "f32"])
@pytest.mark.parametrize("shape", TC_SHAPES)
def test_tc_sketch_matches_oracle(tdk, ctx, shape, dtype):
    ranks = [min(5, s - 2) for s in shape]
    p = 2
    Y, W, _ = small_problem(shape, ranks, p, seed=13, dtype=dtype)
    U, Z = tdk.tucker_sketch(ctx, dev_tensor(Y, dtype), dev_W(W), ranks, p, "tc", want_Z=True)
    assert ctx.sync_status() == 0
    Zo, _ = oracle.sketch(Y, W)
    bnd = sketch_abs_bound(Y, W)
    N = len(shape)
    for n in range(N):
        tol = _tc_tol(dtype, n == N - 1, ranks[-1] + p)
        err = np.abs(host(Z[n]) - Zo[n])
        assert np.all(err <= tol * bnd[n] + 1e-30), (n, float((err / bnd[n]).max()), tol)


@pytest.mark.parametrize("dtype", ["bf16", "f32"])
@pytest.mark.parametrize("shape,ranks", [((40, 130, 264), (20, 18, 22)), ((48, 200, 256), (40, 38, 44)),
                                         ((6, 9, 140, 136), (4, 7, 26, 30))])
def test_tc_sketch_wide_ranks_matches_oracle(tdk, ctx, shape, ranks, dtype):
    # sketch widths 17..32 and above 32: every channel block of the epilogue
    # (both warp groups, all K_p chunks) carries data
    p = 2
    Y, W, _ = small_problem(shape, ranks, p, seed=14, dtype=dtype)
    U, Z = tdk.tucker_sketch(ctx, dev_tensor(Y, dtype), dev_W(W), ranks, p, "tc", want_Z=True)
    assert ctx.sync_status() == 0
    Zo, _ = oracle.sketch(Y, W)
    bnd = sketch_abs_bound(Y, W)
    N = len(shape)
    for n in range(N):
        tol = _tc_tol(dtype, n == N - 1, ranks[-1] + p)
        err = np.abs(host(Z[n]) - Zo[n])
        assert np.all(err <= tol * bnd[n] + 1e-30), (n, float((err / bnd[n]).max()), tol)


@pytest.mark.parametrize("dtype", ["bf16", "f32"])
@pytest.mark.parametrize("shape,ranks", [((67, 45, 136), (5, 5, 5)), ((40, 130, 264), (20, 20, 20)),
                                         ((48, 200, 256), (40, 40, 40)), ((6, 9, 140, 136), (4, 4, 4, 4)),
                                         ((9, 11, 7, 16), (5, 5, 5, 5))])
def test_tc_sketch_shared_family_matches_oracle(tdk, ctx, shape, ranks, dtype):
    # W_k^(n) = W_k for every n: the kernel contracts the shared last-mode
    # block once for all modes < N-1 (same pointer, same width); the result is
    # the oracle's sketch of the same matrices, and the same as when the
    # shared matrices are passed as separate copies (independent blocks)
    p = 2
    Y, W, _ = small_problem(shape, ranks, p, seed=15, dtype=dtype, shared=True)
    N = len(shape)
    assert all(W[n][N - 1] is W[0][N - 1] for n in range(N - 1))
    Yd = dev_tensor(Y, dtype)
    Zo, _ = oracle.sketch(Y, W)
    bnd = sketch_abs_bound(Y, W)
    copies = [[None if w is None else w.copy() for w in row] for row in W]
    for Win in (dev_W(W), dev_W(copies)):
        U, Z = tdk.tucker_sketch(ctx, Yd, Win, ranks, p, "tc", want_Z=True)
        assert ctx.sync_status() == 0
        for n in range(N):
            tol = _tc_tol(dtype, n == N - 1, ranks[-1] + p)
            err = np.abs(host(Z[n]) - Zo[n])
            assert np.all(err <= tol * bnd[n] + 1e-30), (n, float((err / bnd[n]).max()), tol)


def _tc_core_split(dtype):
    """Relative error bound of the hi + lo splits in the tensor-core core pass
    (each split leaves a residual below 2^-17 of the value).  FP32 data: U_N
    and Y split (2 x 2^-17).  BF16 data (Y exact): U_N, then in the fused
    second contraction X_1 and U_{N-1} (3 x 2^-17)."""
    return 2 * 2.0 ** -17 if dtype == "f32" else 3 * 2.0 ** -17


@pytest.mark.parametrize("dtype", ["bf16", "f32"])
@pytest.mark.parametrize("shape", TC_SHAPES)
def test_tc_core_matches_oracle(tdk, ctx, shape, dtype):
    ranks = [min(5, s - 2) for s in shape]
    p = 2
    Y, W, _ = small_problem(shape, ranks, p, seed=17, dtype=dtype)
    ref = oracle.rand_tucker(Y, W)
    Ud = [dev_tensor(u, "f64") for u in ref["U"]]
    G, nrm = tdk.tucker_core(ctx, dev_tensor(Y, dtype), Ud, ranks, p, "tc")
    assert ctx.sync_status() == 0
    bnd = core_abs_bound(Y, ref["U"])
    tol = 2e-5 + _tc_core_split(dtype)
    err = np.abs(host(G) - ref["G"])
    assert np.all(err <= tol * bnd), float((err / bnd).max())
    assert math.isclose(float(nrm.item()), ref["normY2"], rel_tol=1e-6)


@pytest.mark.parametrize("shape,ranks", [((320, 140, 72), (6, 7, 8)), ((160, 257, 384), (40, 38, 44)),
                                         ((6, 40, 30, 136), (4, 5, 6, 7)), ((200, 128, 64), (3, 60, 60)),
                                         ((600, 40, 64), (10, 12, 14)), ((300, 136, 64), (40, 40, 40))])
def test_tc_core_fused_matches_oracle(tdk, ctx, shape, ranks):
    # BF16 data: the fused first two contractions.  More work items (outer
    # indices) than SMs, ragged and exact 128-row tiles of the second mode,
    # fewer and more 64-column chunks than ring stages, sketch widths from 8
    # to 62, and a 4-way case (outer index over two modes)
    p = 2
    Y, W, _ = small_problem(shape, ranks, p, seed=29, dtype="bf16")
    U = [np.linalg.qr(np.random.default_rng(30 + n).standard_normal((I, r + p)))[0]
         for n, (I, r) in enumerate(zip(shape, ranks))]
    Gref = oracle.tucker_core(Y, U)
    G, nrm = tdk.tucker_core(ctx, dev_tensor(Y, "bf16"), [dev_tensor(u, "f64") for u in U], ranks, p, "tc")
    assert ctx.sync_status() == 0
    bnd = core_abs_bound(Y, U)
    tol = 2e-5 + _tc_core_split("bf16")
    err = np.abs(host(G) - Gref)
    assert np.all(err <= tol * bnd), (shape, float((err / bnd).max()))
    assert math.isclose(float(nrm.item()), float(np.sum(Y.astype(np.float64) ** 2)), rel_tol=1e-6)


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_tc_end_to_end_scaled(tdk, ctx, dtype):
    """Workload 2's data model at 128^3 on the tensor-core form: the
    reconstruction error differs from the oracle's by <= 1e-5 (FP32 data) or
    <= 1e-3 (BF16 data)."""
    w = synth.scaled(synth.WORKLOADS["c2"], (128, 128, 128))
    w.dtype = dtype
    Y = synth.host_tensor(w)
    W = synth.sketch_matrices(w.shape, w.Rt, w.seed)
    ref = oracle.rand_tucker(Y, W)
    Yd = dev_tensor(Y, dtype)
    U, _ = tdk.tucker_sketch(ctx, Yd, dev_W(W), w.ranks, w.p, "tc")
    G, nrm = tdk.tucker_core(ctx, Yd, U, w.ranks, w.p, "tc")
    e_gpu = recon_err(float(nrm.item()), host(G))
    e_or = recon_err(ref["normY2"], ref["G"])
    assert abs(e_gpu - e_or) <= (1e-5 if dtype == "f32" else 1e-3), (e_gpu, e_or)


@pytest.mark.parametrize("cfg", ["c4", "c2"])
def test_full_size_sketch_rows_match_oracle(tdk, ctx, cfg):
    """The bench workloads at full size (3000^3 BF16, 1000^3 FP32) through
    the bench's tensor-core path: sampled rows Z_n[i, :] against the oracle's
    row-by-row sketch of the same slab, with the tolerance of the small-size
    tests; U_n orthonormal; ||G|| <= ||Y|| (orthogonal projection)."""
    import torch

    w = synth.WORKLOADS[cfg]
    N = len(w.shape)
    Y, _ = synth.device_tensor(w, device="cuda")
    W = synth.sketch_matrices(w.shape, w.Rt, w.seed)
    Wabs = [[None if x is None else np.abs(x) for x in row] for row in W]
    try:
        U, Z = tdk.tucker_sketch(ctx, Y, dev_W(W), w.ranks, w.p, "tc", want_Z=True)
        G, nrm = tdk.tucker_core(ctx, Y, U, w.ranks, w.p, "tc")
        assert ctx.sync_status() == 0
        rng = np.random.default_rng(7)
        for n in range(N):
            tol = _tc_tol(w.dtype, n == N - 1, w.Rt[-1])
            rows = [0, w.shape[n] - 1] + [int(i) for i in rng.choice(w.shape[n], 2, replace=False)]
            Zn = host(Z[n])
            for i in rows:
                idx = [slice(None)] * N
                idx[n] = i
                slab = Y[tuple(idx)].to(torch.float64).cpu().numpy()
                ref = oracle.sketch_row(slab, n, W)
                bnd = oracle.sketch_row(np.abs(slab), n, Wabs)
                err = np.abs(Zn[i] - ref)
                assert np.all(err <= tol * bnd + 1e-30), (cfg, n, i, float((err / bnd).max()), tol)
            Un = host(U[n])
            assert np.abs(Un.T @ Un - np.eye(Un.shape[1])).max() < 1e-12
        g2 = float(np.sum(host(G) ** 2))
        assert 0.0 < g2 <= float(nrm.item()) * (1.0 + 1e-5)
    finally:
        del Y
        torch.cuda.empty_cache()


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_matrix_case_matches_oracle(tdk, ctx, dtype, als_form):
    """N = 2 (a matrix): the sketches are Y W and Y^T W, the core U_1^T Y U_2,
    and FFCP is ALS on that small matrix.  Both ALS forms (the persistent
    kernel hands N = 2 to the kernel-per-step form)."""
    shape, ranks, p, R = (90, 70), (6, 5), 3, 4
    Y, W, _ = small_problem(shape, ranks, p, seed=41, dtype=dtype, R_cp=R)
    Yd = dev_tensor(Y, dtype)
    U, Z = tdk.tucker_sketch(ctx, Yd, dev_W(W), ranks, p, "simt", want_Z=True)
    Zo, _ = oracle.sketch(Y, W)
    bnd = sketch_abs_bound(Y, W)
    for n in range(2):
        err = np.abs(host(Z[n]) - Zo[n])
        assert np.all(err <= TOL_SKETCH[(dtype, "simt")] * bnd[n] + 1e-300), n
    Uh = [host(u) for u in U]
    G, nrm = tdk.tucker_core(ctx, Yd, U, ranks, p, "simt")
    Gref = oracle.tucker_core(Y, Uh)
    tol = 1e-12 if dtype == "f64" else 2e-5
    assert np.all(np.abs(host(G) - Gref) <= tol * core_abs_bound(Y, Uh))
    Rt = [r + p for r in ranks]
    B0 = synth.init_factors(Rt, R, 5)
    ref_als = oracle.cp_als(Gref, B0, max_sweeps=40, tol=0.0)
    out = tdk.ffcp_als(ctx, G, U, shape, ranks, p, DT_CODE[dtype], R, max_sweeps=40, tol=0.0,
                       B0=[dev_tensor(b, "f64") for b in B0], normY2=nrm)
    assert ctx.sync_status() == 0
    assert out["sweeps"] == 40
    assert abs(out["fit_core"] - ref_als["fit"]) < (1e-9 if dtype == "f64" else 1e-5)


@pytest.mark.parametrize("prec,dtype", [("simt", "f64"), ("simt", "f32"), ("tc", "f32"), ("tc", "bf16")])
def test_full_width_sketch_reconstructs_exactly(tdk, ctx, prec, dtype):
    """Degenerate width R_n + p = I_n: every U_n is a square orthogonal
    matrix, so the Tucker model reproduces Y and ||G|| = ||Y||."""
    shape, ranks, p = (20, 24, 32), (18, 22, 30), 2
    Y, W, _ = small_problem(shape, ranks, p, seed=43, dtype=dtype)
    Yd = dev_tensor(Y, dtype)
    U, _ = tdk.tucker_sketch(ctx, Yd, dev_W(W), ranks, p, prec)
    G, nrm = tdk.tucker_core(ctx, Yd, U, ranks, p, prec)
    assert ctx.sync_status() == 0
    Uh = [host(u) for u in U]
    for u in Uh:
        assert u.shape[0] == u.shape[1]
        assert np.abs(u.T @ u - np.eye(u.shape[0])).max() < 1e-12
    Yr = oracle.tucker_full(host(G), Uh)
    rel = np.linalg.norm(Yr - Y) / np.linalg.norm(Y)
    assert rel < (1e-12 if dtype == "f64" else (2e-5 if prec == "simt" else 1e-4)), rel
    assert math.isclose(float(np.sum(host(G) ** 2)), float(nrm.item()),
                        rel_tol=1e-11 if dtype == "f64" else (1e-4 if prec == "simt" else 5e-4))


def test_tensor_core_form_rejects_what_it_does_not_cover(tdk, ctx):
    """N = 2 and FP64 data have no tensor-core form: TDK_ENOTSUP, nothing run."""
    Y, W, _ = small_problem((40, 32), (4, 4), 2, seed=45, dtype="f32")
    with pytest.raises(tdk.TdkError):
        tdk.tucker_sketch(ctx, dev_tensor(Y, "f32"), dev_W(W), (4, 4), 2, "tc")
    Y3, W3, _ = small_problem((12, 10, 16), (3, 3, 3), 2, seed=46, dtype="f64")
    with pytest.raises(tdk.TdkError):
        tdk.tucker_sketch(ctx, dev_tensor(Y3, "f64"), dev_W(W3), (3, 3, 3), 2, "tc")
    assert ctx.sync_status() == 0


def test_host_data_through_the_abi_copies(tdk, ctx):
    """decompose on a host tensor (copied in by tdk_copy_in) gives the same
    result as on the device tensor; tdk_copy_out returns the factors."""
    import torch

    shape, ranks, p, R = (40, 36, 48), (4, 4, 4), 2, 3
    Y, W, _ = small_problem(shape, ranks, p, seed=47, dtype="f32")
    Yh = torch.as_tensor(Y, dtype=torch.float32).pin_memory()
    Yd = Yh.to("cuda")
    Wd = dev_W(W)
    B0 = [dev_tensor(b, "f64") for b in synth.init_factors([r + p for r in ranks], R, 3)]
    a = tdk.decompose(ctx, Yd, Wd, ranks, p, R, "tc", max_sweeps=30, tol=0.0, B0=B0)
    buf = torch.empty_like(Yd)
    b = tdk.decompose(ctx, Yh, Wd, ranks, p, R, "tc", max_sweeps=30, tol=0.0, B0=B0, Y_dev=buf)
    assert torch.equal(buf, Yd)
    for n in range(3):
        ha = tdk.copy_out(ctx, a["A"][n])
        hb = tdk.copy_out(ctx, b["A"][n])
        assert ha.device.type == "cpu" and torch.equal(ha, hb)
    assert a["fit_core"] == b["fit_core"]
    assert ctx.sync_status() == 0


@pytest.mark.parametrize("pinned,offset,extra", [(True, 0, 5), (True, 8, 0), (False, 0, 3), (True, 0, -(1 << 25))])
def test_copy_in_every_path_is_exact(tdk, ctx, pinned, offset, extra):
    """tdk_copy_in: a page-locked 16-byte-aligned source of 64 MiB or more
    goes through the SM copy kernel (with its tail bytes by the copy engine);
    an unaligned, a pageable or a smaller source goes through the copy
    engine.  Every path delivers the bytes exactly."""
    import torch

    n = (1 << 26) + extra
    src = torch.randint(0, 256, (n + offset,), dtype=torch.uint8)
    if pinned:
        src = src.pin_memory()
    view = src[offset:]
    dst = torch.empty(n, dtype=torch.uint8, device="cuda")
    tdk.copy_in(ctx, dst, view)
    torch.cuda.synchronize()
    assert ctx.sync_status() == 0
    assert torch.equal(dst.cpu(), view)


@pytest.mark.parametrize("rule", ["hals", "mu"])
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_nonneg_rules_match_oracle(tdk, ctx, rule, dtype):
    """HALS (Eq. 8) and multiplicative (Eq. 15) nonnegative FFCP in the
    persistent kernel against the oracle's rules on the same 4-way core."""
    shape, ranks, p, R = (24, 22, 20, 18), (5, 5, 5, 5), 3, 4
    Y, W, A = small_problem(shape, ranks, p, seed=7, dtype="f64", snr=25.0, R_cp=R, dist="uniform", clip0=True)
    ref = oracle.rand_tucker(Y, W)
    A0 = synth.init_factors(shape, R, 6, dist="uniform")
    o = oracle.cp_als_nonneg(ref["G"], ref["U"], A0, max_sweeps=40, tol=0.0, rule=rule)
    out = tdk.ffcp_als(ctx, dev_tensor(ref["G"], dtype), [dev_tensor(u, "f64") for u in ref["U"]], shape, ranks,
                       p, DT_CODE[dtype], R, max_sweeps=40, tol=0.0, nonneg=rule,
                       A0=[dev_tensor(a, "f64") for a in A0])
    assert ctx.sync_status() == 0
    assert out["sweeps"] == 40
    assert abs(out["fit_core"] - o["fit"]) < (1e-10 if dtype == "f64" else 1e-5), (out["fit_core"], o["fit"])
    Ah = [host(a) for a in out["A"]]
    assert all(np.all(a >= 0) for a in Ah)
    Ao = [a.copy() for a in o["A"]]
    Ao[-1] = Ao[-1] * o["lam"][None, :]
    if dtype == "f64":
        for n in range(4):
            assert np.allclose(Ah[n], Ao[n], atol=1e-8)
    else:
        assert oracle.congruence(Ao, Ah) > 0.9999


@pytest.mark.parametrize("rule", ["hals", "mu", "l1", "l1+"])
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_nonneg_rules_in_the_steps_form_match_oracle(tdk, ctx, rule, dtype):
    """HALS (Eq. 8), MU (Eq. 15) and the l1 update (Eq. 16, signed and
    projected) in the kernel-per-step form, the form that takes factors whose
    rows do not fit on chip, against the oracle's rules on the same core."""
    shape, ranks, p, R = (24, 22, 20, 18), (5, 5, 5, 5), 3, 4
    clip = rule != "l1"
    dist = "uniform" if clip else "normal"
    Y, W, _ = small_problem(shape, ranks, p, seed=8, dtype="f64", snr=25.0, R_cp=R, dist=dist, clip0=clip)
    ref = oracle.rand_tucker(Y, W)
    A0 = synth.init_factors(shape, R, 6, dist=dist)
    c = 0.05 if rule.startswith("l1") else 0.0
    orule = rule if rule in ("hals", "mu") else "ls"
    o = oracle.cp_als_nonneg(ref["G"], ref["U"], A0, max_sweeps=25, tol=0.0, rule=orule, l1=c, clip=clip)
    nn = rule if rule in ("hals", "mu") else ("ls" if clip else False)
    out = tdk.ffcp_als(ctx, dev_tensor(ref["G"], dtype), [dev_tensor(u, "f64") for u in ref["U"]], shape, ranks,
                       p, DT_CODE[dtype], R, max_sweeps=25, tol=0.0, nonneg=nn,
                       A0=[dev_tensor(a, "f64") for a in A0], l1=c, form="steps")
    assert out["form"] == "steps"
    assert ctx.sync_status() == 0
    assert out["sweeps"] == 25
    assert abs(out["fit_core"] - o["fit"]) < (1e-10 if dtype == "f64" else 1e-5)
    Ah = [host(a) for a in out["A"]]
    if clip:
        assert all(np.all(a >= 0) for a in Ah)
    Ao = [a.copy() for a in o["A"]]
    Ao[-1] = Ao[-1] * o["lam"][None, :]
    if dtype == "f64":
        for n in range(4):
            assert np.allclose(Ah[n], Ao[n], atol=1e-8)
    else:
        assert oracle.congruence(Ao, Ah) > 0.9999


@pytest.mark.parametrize("clip", [False, True])
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_l1_rule_matches_oracle(tdk, ctx, clip, dtype):
    """The l1-regularised update of Eq. 16 (soft threshold of the LS rows,
    signed or projected) against the oracle on the same core."""
    shape, ranks, p, R = (24, 22, 20), (5, 5, 5), 3, 4
    dist = "uniform" if clip else "normal"
    Y, W, _ = small_problem(shape, ranks, p, seed=9, dtype="f64", snr=25.0, R_cp=R, dist=dist, clip0=clip)
    ref = oracle.rand_tucker(Y, W)
    A0 = synth.init_factors(shape, R, 6, dist=dist)
    c = 0.05
    o = oracle.cp_als_nonneg(ref["G"], ref["U"], A0, max_sweeps=30, tol=0.0, l1=c, clip=clip)
    out = tdk.ffcp_als(ctx, dev_tensor(ref["G"], dtype), [dev_tensor(u, "f64") for u in ref["U"]], shape, ranks,
                       p, DT_CODE[dtype], R, max_sweeps=30, tol=0.0, nonneg="ls" if clip else False,
                       A0=[dev_tensor(a, "f64") for a in A0], l1=c)
    assert ctx.sync_status() == 0
    assert out["sweeps"] == 30
    assert abs(out["fit_core"] - o["fit"]) < (1e-10 if dtype == "f64" else 1e-4), (out["fit_core"], o["fit"])
    if dtype == "f64":
        Ah = [host(a) for a in out["A"]]
        Ao = [a.copy() for a in o["A"]]
        Ao[-1] = Ao[-1] * o["lam"][None, :]
        for n in range(3):
            assert np.allclose(Ah[n], Ao[n], atol=1e-8)
        if clip:
            assert all(np.all(a >= 0) for a in Ah)


@pytest.mark.parametrize("nonneg", [False, True])
def test_ffcp_on_tucker_format_input_at_large_dimension(tdk, ctx, nonneg):
    """FFCP on a Tucker-format input with I_n = 10^4 and no dense Y (the
    large-dimension experiment of Sec. V): a planted CP model is given by its
    core and orthonormal factors; the lifted factors are compared with the
    oracle's (unconstrained: the core-space ALS lifted; nonneg: the
    ambient-row form, whose rows do not fit on chip and take the
    kernel-per-step form)."""
    I, Rt, R = 10000, 8, 3
    shape, ranks, p = (I, I, I), (Rt - 2, Rt - 2, Rt - 2), 2
    r_ = np.random.default_rng(51)
    U = [np.linalg.qr(r_.standard_normal((I, Rt)))[0] for _ in range(3)]
    if nonneg:
        # a nonnegative planted model inside the span of U: A_n = |U_n C_n| projected back
        C = [np.abs(r_.standard_normal((Rt, R))) for _ in range(3)]
        A = [np.abs(u @ c) for u, c in zip(U, C)]
        U = [np.linalg.qr(np.concatenate([a, r_.standard_normal((I, Rt - R))], axis=1))[0] for a in A]
        B = [u.T @ a for u, a in zip(U, A)]
    else:
        B = [r_.standard_normal((Rt, R)) for _ in range(3)]
    G = oracle.cp_full(np.ones(R), B) + 1e-3 * r_.standard_normal((Rt, Rt, Rt))
    Gd = dev_tensor(G, "f64")
    Ud = [dev_tensor(u, "f64") for u in U]
    if nonneg:
        A0 = [np.abs(r_.standard_normal((I, R))) for _ in range(3)]
        o = oracle.cp_als_nonneg(G, U, A0, max_sweeps=25, tol=0.0)
        out = tdk.ffcp_als(ctx, Gd, Ud, shape, ranks, p, 0, R, max_sweeps=25, tol=0.0, nonneg=True,
                           A0=[dev_tensor(a, "f64") for a in A0])
        Ao = [a.copy() for a in o["A"]]
        Ao[-1] = Ao[-1] * o["lam"][None, :]
    else:
        B0 = [r_.standard_normal((Rt, R)) for _ in range(3)]
        o = oracle.cp_als(G, B0, max_sweeps=25, tol=0.0)
        out = tdk.ffcp_als(ctx, Gd, Ud, shape, ranks, p, 0, R, max_sweeps=25, tol=0.0,
                           B0=[dev_tensor(b, "f64") for b in B0])
        Ao = oracle.lift(U, o["B"], o["lam"])
    assert ctx.sync_status() == 0
    assert abs(out["fit_core"] - o["fit"]) < 1e-10
    Ah = [host(a) for a in out["A"]]
    assert all(a.shape == (I, R) for a in Ah)
    for n in range(3):
        assert np.allclose(Ah[n], Ao[n], atol=1e-8)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("shape,ranks", [((40, 36, 32), (5, 6, 7)), ((14, 12, 10, 16), (3, 4, 3, 5))])
def test_rand_tucker_2i_matches_oracle(tdk, ctx, dtype, shape, ranks):
    """RandTucker2i (Alg. 3): two refinement passes from Gaussian factors,
    then the core, against the oracle on the same inputs."""
    p = 2
    Rt = [r + p for r in ranks]
    Y, _, _ = small_problem(shape, ranks, p, seed=53, dtype=dtype)
    U0 = synth.random_factors(shape, Rt, 53)
    Wp = [synth.refine_matrices(Rt, 53, it) for it in range(2)]
    ref = oracle.rand_tucker_2i(Y, U0, Wp)
    U, G, nrm = tdk.rand_tucker_2i(ctx, dev_tensor(Y, dtype), [dev_tensor(u, "f64") for u in U0],
                                   [dev_W(W) for W in Wp], ranks, p)
    assert ctx.sync_status() == 0
    Uh = [host(u) for u in U]
    for u in Uh:
        assert np.abs(u.T @ u - np.eye(u.shape[1])).max() < 1e-12
    if dtype == "f64":
        for n in range(len(shape)):
            assert np.abs(Uh[n] - ref["U"][n]).max() < 1e-8, n
        bnd = core_abs_bound(Y, ref["U"])
        assert np.all(np.abs(host(G) - ref["G"]) <= 1e-9 * bnd)
    else:
        e_gpu = recon_err(float(nrm.item()), host(G))
        e_or = recon_err(ref["normY2"], ref["G"])
        assert abs(e_gpu - e_or) <= 1e-5, (e_gpu, e_or)
