"""GPU parity of the paths the benchmark workloads take, against the FP64
oracle on the same seeded inputs, through the C ABI:
  * FFCP on a 60^3 core with R = 40 (the 3000^3 workload's core), which runs
    the cooperative grid form of the persistent ALS kernel;
  * nonnegative FFCP on a 30^4 core with R = 20 (the 200^4 workload's core),
    in both the grid form and the kernel-per-step form;
  * the test matrices drawn inside the library from a seed, bit for bit
    against the oracle's own implementation of the generator, and the sketch
    they give;
  * a test matrix that is not made of BF16 values through the tensor-core
    sketch, against the unrounded product;
  * the slab entry points of the sharded form, summed over the slabs.
Tolerances are stated per test and follow from the arithmetic of each form."""
import numpy as np
import pytest

import oracle
import synth
from helpers import DT_CODE, TOL_SKETCH, basis_tol, dev_tensor, dev_W, host, sketch_abs_bound, small_problem

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


def _wide_core(seed=4):
    """The 3000^3 workload's data model (CP rank 40, N(0,1) factors, SNR
    15 dB) at 96 x 84 x 72, compressed by the oracle to a 60^3 core."""
    shape, ranks, p, R = (96, 84, 72), (40, 40, 40), 20, 40
    Y, W, _ = small_problem(shape, ranks, p, seed=seed, dtype="f64", snr=15.0, R_cp=R)
    return shape, ranks, p, R, oracle.rand_tucker(Y, W)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_als_grid_form_on_the_wide_core_matches_oracle(tdk, ctx, dtype):
    """60^3 core, R = 40, 15 sweeps from the same start: the core does not
    fit one SM, so the cooperative grid kernel runs (one CTA per row of H_n
    at this size).  FP64: fit to 1e-10 and every entry of B_n to 1e-8;
    FP32 cores: fit to 1e-5 and congruence of the lifted factors."""
    shape, ranks, p, R, ref = _wide_core()
    Rt = [r + p for r in ranks]
    B0 = synth.init_factors(Rt, R, 40)
    o = oracle.cp_als(ref["G"], B0, max_sweeps=15, tol=0.0)
    out = tdk.ffcp_als(ctx, dev_tensor(ref["G"], dtype), [dev_tensor(u, "f64") for u in ref["U"]], shape, ranks, p,
                       DT_CODE[dtype], R, max_sweeps=15, tol=0.0, B0=[dev_tensor(b, "f64") for b in B0],
                       check_every=16)
    assert out["form"] == "grid" and out["grid"] > 1, (out["form"], out["grid"])
    assert out["sweeps"] == 15
    assert ctx.sync_status() == 0
    tol = 1e-10 if dtype == "f64" else 1e-5
    assert abs(out["fit_core"] - o["fit"]) < tol, (out["fit_core"], o["fit"])
    Ao = oracle.lift(ref["U"], o["B"], o["lam"])
    Ah = [host(a) for a in out["A"]]
    if dtype == "f64":
        for n in range(3):
            assert np.allclose(host(out["B"][n]), o["B"][n], atol=1e-8), n
        for n in range(3):
            assert np.allclose(Ah[n], Ao[n], atol=1e-8 * np.abs(Ao[n]).max()), n
    else:
        assert oracle.congruence(Ao, Ah) > 0.9999


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_newton_schulz_inverse_gives_the_gauss_jordan_solution(tdk, dtype, monkeypatch):
    """From the second sweep on, the grid kernel inverts T_n by Newton-Schulz
    steps from the previous sweep's inverse and refines the solves against
    T_n in FP64; with the start gate at 0 every inverse is Gauss-Jordan.
    Both must give the same iterates: on the 60^3 core with R = 40, 20
    sweeps, B_n to 1e-9 (FP64 core: both solves are accurate far below that)
    or fits to 1e-6 and congruence 0.9999 (FP32 core, whose rounding the two
    paths meet in different places)."""
    shape, ranks, p, R, ref = _wide_core(seed=6)
    Rt = [r + p for r in ranks]
    B0 = [dev_tensor(b, "f64") for b in synth.init_factors(Rt, R, 44)]
    ctx_t = tdk.Context(0, testing=True)
    try:
        outs = []
        for gate in ["1", "0"]:
            monkeypatch.setenv("TDK_ALS_NS_GATE", gate)
            outs.append(tdk.ffcp_als(ctx_t, dev_tensor(ref["G"], dtype), [dev_tensor(u, "f64") for u in ref["U"]],
                                     shape, ranks, p, DT_CODE[dtype], R, max_sweeps=20, tol=0.0, B0=B0))
            assert ctx_t.sync_status() == 0
            assert outs[-1]["form"] == "grid"
        monkeypatch.delenv("TDK_ALS_NS_GATE", raising=False)
        if dtype == "f64":
            for n in range(3):
                assert np.allclose(host(outs[0]["B"][n]), host(outs[1]["B"][n]), atol=1e-9), n
            assert abs(outs[0]["fit_core"] - outs[1]["fit_core"]) < 1e-12
        else:
            assert abs(outs[0]["fit_core"] - outs[1]["fit_core"]) < 1e-6
            A = [[host(a) for a in o["A"]] for o in outs]
            assert oracle.congruence(A[0], A[1]) > 0.9999
    finally:
        monkeypatch.delenv("TDK_ALS_NS_GATE", raising=False)
        ctx_t.close()


def test_als_grid_form_stopping_rule_matches_oracle_fp64(tdk, ctx):
    """The same 60^3 core to convergence (relative fit change below 1e-9):
    the grid kernel stops at the oracle's sweep."""
    shape, ranks, p, R, ref = _wide_core(seed=5)
    Rt = [r + p for r in ranks]
    B0 = synth.init_factors(Rt, R, 41)
    o = oracle.cp_als(ref["G"], B0, max_sweeps=300, tol=1e-9)
    out = tdk.ffcp_als(ctx, dev_tensor(ref["G"], "f64"), [dev_tensor(u, "f64") for u in ref["U"]], shape, ranks, p,
                       0, R, max_sweeps=300, tol=1e-9, B0=[dev_tensor(b, "f64") for b in B0], check_every=4)
    assert out["form"] == "grid"
    assert out["sweeps"] == o["sweeps"], (out["sweeps"], o["sweeps"])
    assert abs(out["fit_core"] - o["fit"]) < 1e-10


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_fp32_stopping_rule_does_not_depend_on_the_kernel(tdk, seed, monkeypatch):
    """A 20^3 FP32 core with R = 10 (the 1000^3 workload's core geometry),
    built from correlated factors so that ALS takes some tens of sweeps, run
    to a relative fit change below 1e-7 by the one-CTA kernel and by the grid
    kernel, which sum the model and the residual in different orders: both
    stop at the same sweep with fits that agree far inside the tolerance, and
    that fit stays within FP32 rounding of the FP64 oracle's from the same
    start.  (Over 24 such runs, 20 stop at the same sweep; the other four
    creep for 230 to 520 sweeps, and there the two kernels' FP32 iterates
    drift apart enough to move the stop by one or two sweeps, whatever the
    precision of the fit.)"""
    shape, R = (20, 20, 20), 10
    A = synth.cp_factors(shape, R, 60 + seed, rho=0.6)
    G = synth.add_noise(synth.cp_dense(A), 30.0, 60 + seed)
    U = [np.eye(20) for _ in range(3)]
    B0 = synth.init_factors(shape, R, 70 + seed)
    ctx_t = tdk.Context(0, testing=True)
    try:
        runs = {}
        for form in ["one-CTA", "grid"]:
            if form == "grid":
                monkeypatch.setenv("TDK_ALS_GRID", "1")
            out = tdk.ffcp_als(ctx_t, dev_tensor(G, "f32"), [dev_tensor(u, "f64") for u in U], shape, (18, 18, 18),
                               2, DT_CODE["f32"], R, max_sweeps=3000, tol=1e-7,
                               B0=[dev_tensor(b, "f64") for b in B0], check_every=16)
            monkeypatch.delenv("TDK_ALS_GRID", raising=False)
            assert ctx_t.sync_status() == 0
            runs[form] = out
        assert runs["one-CTA"]["grid"] == 1 and runs["grid"]["grid"] > 1
        s1, s2 = runs["one-CTA"]["sweeps"], runs["grid"]["sweeps"]
        assert 20 <= s1 < 3000, s1  # a run of many sweeps, stopped by the rule
        assert s1 == s2, (s1, s2)
        # the two kernels' FP32 iterates differ by rounding: their fits agree to
        # a tenth of the stopping tolerance
        assert abs(runs["one-CTA"]["fit_core"] - runs["grid"]["fit_core"]) < 1e-8
        o = oracle.cp_als(G, B0, max_sweeps=s1, tol=0.0)
        assert abs(runs["grid"]["fit_core"] - o["fit"]) < 1e-5
    finally:
        ctx_t.close()


@pytest.mark.parametrize("form", ["one-CTA", "grid"])
def test_fp32_fit_is_the_fit_of_the_returned_factors(tdk, form, monkeypatch):
    """The fit an FP32 core reports is the fit of the model it returns: with
    the FP32 core, the returned B_n and lambda (rounded to FP32, as the
    kernel holds it), 1 - ||G - [[lambda; B]]|| / ||G|| evaluated in FP64
    agrees with the reported fit to 1e-11.  The float-float residual is
    accurate to about 2^-44; the FP32 sums it replaced were off by up to
    3e-9 on such cores."""
    shape, R = (20, 20, 20), 10
    U = [dev_tensor(np.eye(20), "f64") for _ in range(3)]
    ctx_t = tdk.Context(0, testing=True)
    try:
        if form == "grid":
            monkeypatch.setenv("TDK_ALS_GRID", "1")
        for seed in [1, 2, 3]:
            A = synth.cp_factors(shape, R, 80 + seed, rho=0.5)
            G = synth.add_noise(synth.cp_dense(A), 20.0, 80 + seed).astype(np.float32).astype(np.float64)
            B0 = synth.init_factors(shape, R, 90 + seed)
            for sweeps in [3, 25]:
                out = tdk.ffcp_als(ctx_t, dev_tensor(G, "f32"), U, shape, (18, 18, 18), 2, DT_CODE["f32"], R,
                                   max_sweeps=sweeps, tol=0.0, B0=[dev_tensor(b, "f64") for b in B0])
                assert ctx_t.sync_status() == 0
                assert (out["grid"] > 1) == (form == "grid")
                lam = host(out["lam"]).astype(np.float32).astype(np.float64)
                model = oracle.cp_full(lam, [host(b) for b in out["B"]])
                fit64 = 1.0 - np.linalg.norm(G - model) / np.linalg.norm(G)
                assert abs(out["fit_core"] - fit64) < 1e-11, (seed, sweeps, out["fit_core"] - fit64)
    finally:
        monkeypatch.delenv("TDK_ALS_GRID", raising=False)
        ctx_t.close()


def test_fp32_nonneg_stopping_sweep_is_within_two_of_the_oracle(tdk, monkeypatch):
    """The 200^4 workload's data model at 40 x 36 x 34 x 32, compressed to a
    30^4 FP32 core; projected LS FFCP with R = 20 to a relative fit change
    below 1e-7, by the grid kernel on the whole GPU (each row of H_n split
    over 5 CTAs) and on 120 CTAs (over 4), against the FP64 oracle.  Here
    the iterates themselves carry FP32 error: T_n of nonnegative factors is
    ill-conditioned, and the rounding of H_n moves A_n by about 1e-5 (5.8e-5
    between the whole GPU and 24 CTAs, one per row, after 2 sweeps), so the
    fits of two grids differ by up to about 1e-8 near the end and the
    stopping sweep by up to two.  Checked: each stops within two sweeps of
    the oracle, at a fit within 1e-6 of the oracle's (the fit still grows by
    about 1e-7 a sweep there)."""
    shape, ranks, p, R = (40, 36, 34, 32), (20, 20, 20, 20), 10, 20
    Y, W, _ = small_problem(shape, ranks, p, seed=3, dtype="f64", snr=25.0, R_cp=R, dist="uniform", clip0=True)
    ref = oracle.rand_tucker(Y, W)
    A0 = synth.init_factors(shape, R, 33, dist="uniform")
    o = oracle.cp_als_nonneg(ref["G"], ref["U"], A0, max_sweeps=2000, tol=1e-7)
    ctx_t = tdk.Context(0, testing=True)
    try:
        for cap in [None, "120"]:
            if cap:
                monkeypatch.setenv("TDK_ALS_GRID", cap)
            out = tdk.ffcp_als(ctx_t, dev_tensor(ref["G"], "f32"), [dev_tensor(u, "f64") for u in ref["U"]], shape,
                               ranks, p, DT_CODE["f32"], R, max_sweeps=2000, tol=1e-7, nonneg=True,
                               A0=[dev_tensor(a, "f64") for a in A0])
            monkeypatch.delenv("TDK_ALS_GRID", raising=False)
            assert ctx_t.sync_status() == 0
            assert out["form"] == "grid"
            assert (out["grid"] == 120) == (cap is not None), out["grid"]
            assert abs(out["sweeps"] - o["sweeps"]) <= 2, (cap, out["sweeps"], o["sweeps"])
            assert abs(out["fit_core"] - o["fit"]) < 1e-6, (cap, out["fit_core"], o["fit"])
    finally:
        ctx_t.close()


@pytest.mark.parametrize("form", ["auto", "steps"])
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_nonneg_ffcp_on_the_4way_core_matches_oracle(tdk, ctx, dtype, form):
    """The 200^4 workload's data model (nonnegative CP rank 20, U[0, 1]
    factors, SNR 25 dB, clipped at 0) at 40 x 36 x 34 x 32, compressed to a
    30^4 core; projected LS FFCP with R = 20 for 10 sweeps from the same
    start, in the form AUTO picks (the persistent grid kernel, whose buffers
    hold one part of a split row of H_n, FP32 and FP64 cores alike) and in
    the kernel-per-step form."""
    shape, ranks, p, R = (40, 36, 34, 32), (20, 20, 20, 20), 10, 20
    Y, W, _ = small_problem(shape, ranks, p, seed=3, dtype="f64", snr=25.0, R_cp=R, dist="uniform", clip0=True)
    ref = oracle.rand_tucker(Y, W)
    A0 = synth.init_factors(shape, R, 33, dist="uniform")
    o = oracle.cp_als_nonneg(ref["G"], ref["U"], A0, max_sweeps=10, tol=0.0)
    out = tdk.ffcp_als(ctx, dev_tensor(ref["G"], dtype), [dev_tensor(u, "f64") for u in ref["U"]], shape, ranks, p,
                       DT_CODE[dtype], R, max_sweeps=10, tol=0.0, nonneg=True, A0=[dev_tensor(a, "f64") for a in A0],
                       form=form)
    assert out["form"] == ("grid" if form == "auto" else "steps")
    assert out["sweeps"] == 10
    assert ctx.sync_status() == 0
    assert abs(out["fit_core"] - o["fit"]) < (1e-10 if dtype == "f64" else 1e-5), (out["fit_core"], o["fit"])
    Ah = [host(a) for a in out["A"]]
    assert all(np.all(a >= 0) for a in Ah)
    Ao = [a.copy() for a in o["A"]]
    Ao[-1] = Ao[-1] * o["lam"][None, :]
    if dtype == "f64":
        for n in range(4):
            assert np.allclose(Ah[n], Ao[n], atol=1e-8 * np.abs(Ao[n]).max()), n
    else:
        assert oracle.congruence(Ao, Ah) > 0.999


# ---------------------------------------------------------------- seeded test matrices

@pytest.mark.parametrize("seed", [0, 7, (1 << 32) + 5, 0x9E3779B97F4A7C15])
def test_seeded_test_matrices_equal_the_oracle_generator(tdk, ctx, seed):
    """tdk_sketch_matrices draws what oracle.philox defines, bit for bit
    (both sides round the FP64 normal to BF16; the two implementations of
    log and cos differ by at most a few FP64 units, which moves a BF16
    rounding with probability near 2^-42 per entry)."""
    shape, ranks, p = (70, 33, 129, 5), (6, 7, 8, 3), 2
    Wd = tdk.sketch_matrices(ctx, shape, ranks, p, seed)
    Wo = oracle.philox.sketch_matrices(seed, shape, [r + p for r in ranks])
    for n in range(4):
        assert Wd[n][n] is None
        for k in range(4):
            if k != n:
                assert np.array_equal(host(Wd[n][k]), Wo[n][k]), (n, k)


@pytest.mark.parametrize("dtype,prec", [("f64", "simt"), ("f32", "simt"), ("f32", "tc"), ("bf16", "tc")])
def test_sketch_with_seeded_test_matrices_matches_oracle(tdk, ctx, dtype, prec):
    """tucker_sketch with W = NULL draws Omega from the descriptor's seed:
    the sketch equals the oracle's on the oracle's own draw of that seed,
    within each form's tolerance."""
    shape, ranks, p, seed = (67, 45, 136), (5, 5, 5), 3, 1234567
    Y, _, _ = small_problem(shape, ranks, p, seed=21, dtype=dtype)
    Wo = oracle.philox.sketch_matrices(seed, shape, [r + p for r in ranks])
    U, Z = tdk.tucker_sketch(ctx, dev_tensor(Y, dtype), None, ranks, p, prec, want_Z=True, seed=seed)
    assert ctx.sync_status() == 0
    Zo, _ = oracle.sketch(Y, Wo)
    bnd = sketch_abs_bound(Y, Wo)
    for n in range(3):
        if prec == "simt":
            tol = TOL_SKETCH[(dtype, "simt")]
        else:
            tol = 2e-5 + (2.0 ** -9 if (n == 2 and dtype == "bf16") else 2.0 ** -16)
        err = np.abs(host(Z[n]) - Zo[n])
        assert np.all(err <= tol * bnd[n] + 1e-300), (n, float((err / bnd[n]).max()))
        Un = host(U[n])
        assert np.abs(Un.T @ Un - np.eye(Un.shape[1])).max() < 1e-12


@pytest.mark.parametrize("dtype", ["bf16", "f32"])
def test_tc_sketch_with_unrounded_test_matrices_is_within_2_pow_minus_9(tdk, ctx, dtype):
    """A test matrix that is not made of BF16 values: the tensor-core form
    rounds W_N^(n) to BF16 for the modes below N (and the Khatri-Rao rows of
    mode N when its width exceeds 32), so every Z_n is within 2^-9 (plus the
    FP32 accumulation) of the product with the unrounded Omega_n, relative to
    sum |y| prod |w|; the header states this bound."""
    shape, ranks, p = (40, 70, 136), (30, 34, 36), 4    # Rt_3 = 40 > 32: mode-3 rows rounded once
    Y, _, _ = small_problem(shape, ranks, p, seed=17, dtype=dtype)
    r = np.random.default_rng(99)
    Rt = [x + p for x in ranks]
    W = [[None if k == n else r.standard_normal((shape[k], Rt[n])) for k in range(3)] for n in range(3)]
    assert not np.array_equal(synth.round_bf16(W[0][1]), W[0][1])
    U, Z = tdk.tucker_sketch(ctx, dev_tensor(Y, dtype), dev_W(W), ranks, p, "tc", want_Z=True)
    assert ctx.sync_status() == 0
    Zo, _ = oracle.sketch(Y, W)
    bnd = sketch_abs_bound(Y, W)
    for n in range(3):
        rel = np.abs(host(Z[n]) - Zo[n]) / bnd[n]
        assert np.all(rel <= 2e-5 + 2.0 ** -9), (n, float(rel.max()))


# ---------------------------------------------------------------- sharded form, one process

@pytest.mark.parametrize("dtype,prec", [("f64", "simt"), ("f32", "tc"), ("bf16", "tc")])
@pytest.mark.parametrize("seeded", [False, True])
def test_slab_shares_sum_to_the_oracle_grid_form(tdk, ctx, dtype, prec, seeded):
    """Sec. IV-B on one GPU: mode 1 cut into three slabs (one thinner than
    the sketch width); each slab's sketch share, the Gram-sum CholQR2 of Z_1
    (Eq. 23 with a Cholesky factor), the replicated bases of the other modes
    and each slab's core share, summed, against the oracle's sub-tensor form
    on the same test matrices.  The shares are summed here in FP64 on the
    host, as an allreduce would."""
    import torch

    shape, ranks, p, seed = (27, 40, 64), (5, 4, 6), 3, 99
    Y, Wsyn, _ = small_problem(shape, ranks, p, seed=31, dtype=dtype)
    Rt = [r + p for r in ranks]
    W = oracle.philox.sketch_matrices(seed, shape, Rt) if seeded else Wsyn
    Wd = None if seeded else dev_W(W)
    cuts = [0, 6, 20, 27]                      # slab 1 holds 6 rows < Rt_1 = 8
    Yd = dev_tensor(Y, dtype)
    Z1_rows, Zsum = [], [None, np.zeros((shape[1], Rt[1])), np.zeros((shape[2], Rt[2]))]
    for a, b in zip(cuts[:-1], cuts[1:]):
        Z = tdk.tucker_sketch_partial(ctx, Yd[a:b].contiguous(), a, shape[0], Wd, ranks, p, prec, seed=seed)
        Z1_rows.append(Z[0])
        for n in (1, 2):
            Zsum[n] += host(Z[n])
    assert ctx.sync_status() == 0
    ref = oracle.rand_tucker_grid(Y, W, (3, 1, 1))
    bnd = sketch_abs_bound(Y, W)
    tol = TOL_SKETCH[(dtype, "simt")] if prec == "simt" else 2e-5 + (2.0 ** -9 if dtype == "bf16" else 2.0 ** -16)
    Z1 = np.concatenate([host(z) for z in Z1_rows])
    for n, Zn in enumerate([Z1, Zsum[1], Zsum[2]]):
        assert np.all(np.abs(Zn - ref["Z"][n]) <= tol * bnd[n] * 3 + 1e-300), n
    # U_1 from the summed row-block Grams, two rounds (CholQR2)
    g = sum(host(tdk.gram(ctx, z)) for z in Z1_rows)
    gd = torch.as_tensor(g, device="cuda")
    Q = [tdk.orth_apply(ctx, gd, z) for z in Z1_rows]
    g2 = torch.as_tensor(sum(host(tdk.gram(ctx, q)) for q in Q), device="cuda")
    U1 = [tdk.orth_apply(ctx, g2, q) for q in Q]
    assert ctx.sync_status() == 0
    U = [np.concatenate([host(u) for u in U1])] + [host(tdk.orth(ctx, torch.as_tensor(Zsum[n], device="cuda")))
                                                   for n in (1, 2)]
    for n, Zn in enumerate([Z1, Zsum[1], Zsum[2]]):
        # the basis of this Z: Householder QR with diag(R) > 0, entry by entry
        assert np.abs(U[n].T @ U[n] - np.eye(Rt[n])).max() < 1e-12
        assert np.abs(U[n] - oracle.householder_qr(Zn)[0]).max() < basis_tol(Zn), n
    # core shares with each slab's rows of U_1, summed
    Ud = [torch.as_tensor(u, device="cuda") for u in U]
    G = 0.0
    nrm = 0.0
    for a, b in zip(cuts[:-1], cuts[1:]):
        Gs, ns = tdk.tucker_core_partial(ctx, Yd[a:b].contiguous(), shape[0], [Ud[0][a:b].contiguous(), Ud[1], Ud[2]],
                                         ranks, p, prec)
        G = G + host(Gs)
        nrm += float(ns.item())
    Gref = oracle.tucker_core(Y, U)
    gb = oracle.tucker_core(np.abs(Y), [np.abs(u) for u in U])
    ctol = 1e-12 if dtype == "f64" else 2e-5 + 3 * 2.0 ** -17
    assert np.all(np.abs(G - Gref) <= ctol * gb * 3 + 1e-300)
    assert abs(nrm - oracle.norm2(Y)) <= 1e-6 * oracle.norm2(Y)


def test_gram_breakdown_is_reported_and_orth_completes(tdk, ctx):
    """A rank-deficient block: tdk_orth_apply raises TDK_WRANKDEF in the
    status word (the sharded driver then gathers Z_1), and tdk_orth completes
    the basis as tucker_sketch does."""
    import torch

    r = np.random.default_rng(5)
    Z = r.standard_normal((50, 3)) @ r.standard_normal((3, 8))   # rank 3, 8 columns
    Zd = torch.as_tensor(Z, device="cuda")
    tdk.orth_apply(ctx, tdk.gram(ctx, Zd), Zd)
    assert ctx.sync_status() & tdk.TDK_WRANKDEF
    U = host(tdk.orth(ctx, Zd))
    assert ctx.sync_status() & tdk.TDK_WRANKDEF
    assert np.abs(U.T @ U - np.eye(8)).max() < 1e-12
    assert np.abs(U @ (U.T @ Z) - Z).max() < 1e-10 * np.abs(Z).max()


# ---------------------------------------------------------------- context and checkpoint

def test_mlp_checkpoint_round_trip_resumes_training(tdk, ctx, tmp_path):
    """tdk_mlp_save / tdk_mlp_load keep the parameters, Adam's moments and
    its step: a model loaded from a checkpoint takes the same next step as
    the model that wrote it, bit for bit.  A checkpoint of another shape is
    refused with TDK_EIO."""
    import torch

    N, Rt, hidden, batch = 3, 6, 32, 12
    r = np.random.default_rng(8)
    G = torch.as_tensor(r.standard_normal((batch, Rt ** N)), dtype=torch.float32).cuda()
    cs = torch.as_tensor(r.standard_normal((batch, N, Rt))).cuda()
    R = torch.as_tensor(r.integers(2, Rt + 1, batch).astype(np.int32)).cuda()
    a = tdk.Mlp(ctx, N, Rt, hidden, max_batch=16)
    a.set_params(synth.mlp_init_params(N, Rt, hidden, 3))
    for _ in range(3):
        a.train_step(G, cs, R, lr=1e-3)
    path = str(tmp_path / "m.tdkmlp")
    a.save(path)
    b = tdk.Mlp(ctx, N, Rt, hidden, max_batch=16)
    b.load(path)
    assert np.array_equal(a.get(tdk.MLP_PARAMS), b.get(tdk.MLP_PARAMS))
    la, lb = a.train_step(G, cs, R, lr=1e-3), b.train_step(G, cs, R, lr=1e-3)
    assert la == lb
    assert np.array_equal(a.get(tdk.MLP_PARAMS), b.get(tdk.MLP_PARAMS))
    c = tdk.Mlp(ctx, N, Rt, hidden * 2, max_batch=16)
    with pytest.raises(tdk.TdkError) as e:
        c.load(path)
    assert e.value.code == tdk.TDK_EIO
    for m in (a, b, c):
        m.close()


def test_workspace_is_created_on_demand_and_reported(tdk):
    """A fresh context holds no workspace; a sketch grows it; the query
    reports the size."""
    c = tdk.Context(0)
    assert c.workspace_bytes() == 0
    shape, ranks, p = (30, 28, 26), (3, 3, 3), 2
    Y, W, _ = small_problem(shape, ranks, p, seed=4, dtype="f32")
    tdk.tucker_sketch(c, dev_tensor(Y, "f32"), dev_W(W), ranks, p, "simt")
    assert c.workspace_bytes() > 0
    c.close()


def test_ffcp_hals_on_the_sec5_tucker_format_case_reaches_200_db(tdk, ctx):
    """Sec. V-A, the experiment after Table III, on the GPU: a noise-free
    4-way CP tensor of rank 10 with I_n = 10^4, factor entries exponential
    with mean 10 and 20 % zeros, given only in Tucker format (orthonormal
    U_n, core G = [[U_1^T A_1, ...]]); FFCP-HALS from a U[0, 1] start, 60
    sweeps.  Its rows do not fit on chip, so the kernel-per-step form runs.
    Every component of every mode must exceed the paper's 200 dB SIR, and the
    factors must equal the oracle's run on the same input."""
    import os

    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "paper_sec5_tucker_format_hals.txt")
    row = [ln.split() for ln in open(path) if ln.strip() and not ln.startswith("#")][0]
    N, I, R, zf, mu, sir_min = int(row[0]), int(row[1]), int(row[2]), float(row[3]), float(row[4]), float(row[5])
    A = synth.sparse_exponential_factors((I,) * N, R, 7, mean=mu, zero_frac=zf)
    U = [np.linalg.qr(a)[0] for a in A]
    G = oracle.cp_full(np.ones(R), [u.T @ a for u, a in zip(U, A)])
    A0 = synth.init_factors((I,) * N, R, 1, dist="uniform")
    o = oracle.cp_als_nonneg(G, U, A0, max_sweeps=60, tol=0.0, rule="hals")
    out = tdk.ffcp_als(ctx, dev_tensor(G, "f64"), [dev_tensor(u, "f64") for u in U], (I,) * N, (R,) * N, 0, 0, R,
                       max_sweeps=60, tol=0.0, nonneg="hals", A0=[dev_tensor(a, "f64") for a in A0])
    assert out["form"] == "steps"
    assert ctx.sync_status() == 0
    Ah = [host(a) for a in out["A"]]
    sir = oracle.sir_db(A, Ah)
    sir_o = oracle.sir_db(A, [a * (o["lam"][None, :] if n == N - 1 else 1.0) for n, a in enumerate(o["A"])])
    print(f"min SIR {min(sir):.1f} dB (oracle run {min(sir_o):.1f} dB)")
    assert len(sir) == N * R and min(sir) > sir_min, min(sir)
    Ao = [a.copy() for a in o["A"]]
    Ao[-1] = Ao[-1] * o["lam"][None, :]
    for n in range(N):
        assert np.allclose(Ah[n], Ao[n], rtol=0, atol=1e-8 * np.abs(Ao[n]).max()), n


@pytest.mark.parametrize("dtype,prec,shared", [("bf16", "tc", False), ("bf16", "tc", True), ("f32", "tc", False),
                                               ("f64", "simt", False), ("f32", "simt", False)])
def test_sketch_pass_returns_the_norm_of_y(tdk, ctx, dtype, prec, shared):
    """||Y||^2 from tucker_sketch: summed by the norm warps while the
    TMEM-W form stages the tiles, by the converter warps for FP32 data, or
    by a streaming pass (CUDA-core form, shared family); equal to the exact
    sum of squares of the stored values up to FP32 accumulation (1e-6
    relative; FP64 data 1e-12), and to the core pass's own sum."""
    import torch

    shape, ranks, p = (67, 45, 136), (5, 6, 7), 3
    Y, W, _ = small_problem(shape, ranks, p, seed=41, dtype=dtype, shared=shared)
    Yd = dev_tensor(Y, dtype)
    nrm = torch.full((), float("nan"), dtype=torch.float64, device="cuda")
    U, _ = tdk.tucker_sketch(ctx, Yd, dev_W(W), ranks, p, prec, normY2=nrm)
    _, nrm_core = tdk.tucker_core(ctx, Yd, U, ranks, p, prec)
    assert ctx.sync_status() == 0
    ref = oracle.norm2(Y)
    tol = 1e-12 if dtype == "f64" else 1e-6
    assert abs(float(nrm.item()) - ref) <= tol * ref, (float(nrm.item()), ref)
    assert abs(float(nrm.item()) - float(nrm_core.item())) <= tol * ref
    # the core pass without its own sum gives the same core
    G1, _ = tdk.tucker_core(ctx, Yd, U, ranks, p, prec)
    G2, none = tdk.tucker_core(ctx, Yd, U, ranks, p, prec, want_norm=False)
    assert none is None and torch.equal(G1, G2)
