"""GPU parity of the learned initialiser (tcgen05 GEMM, canonicalisation,
loss and gradients, Adam, prediction) against the FP64 oracle (oracle/mlp.py)
on the same seeded inputs, through the C ABI.

Tolerances: GEMM products of BF16 values are exact in FP32, so an FP32 output
differs from the FP64 sum by the FP32 accumulation only (bounded by
K * 2^-23 * sum |a b|).  A BF16 output may differ by one BF16 unit
(2^-7 relative) where the pre-rounding values straddle a rounding boundary.
Through the network, such single-unit differences of a few stored
activations bound the norm-wise differences stated per test."""
import ctypes

import numpy as np
import pytest

import oracle
import synth
from oracle import mlp as omlp
from helpers import bf16_ulp, dev_tensor, dev_W, host

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


def _ru8(x):
    return (x + 7) // 8 * 8


def _bf16_dev(X, ld):
    """Row-major BF16 device matrix with leading dimension ld; the padding
    columns hold NaN so that any read outside the matrix shows."""
    import torch

    rows, cols = X.shape
    buf = torch.full((rows, ld), float("nan"), dtype=torch.float32)
    buf[:, :cols] = torch.as_tensor(X, dtype=torch.float32)
    return buf.to(torch.bfloat16).cuda()


GEMM_SHAPES = [(200, 150, 96), (37, 300, 1000), (128, 128, 64), (1, 70, 27), (130, 1200, 256)]


@pytest.mark.parametrize("a_mn,b_mn", [(0, 0), (0, 1), (1, 1), (1, 0)])
@pytest.mark.parametrize("shape", GEMM_SHAPES)
def test_gemm_bf16_layouts_and_epilogues(tdk, ctx, shape, a_mn, b_mn):
    import torch

    M, N, K = shape
    r = np.random.default_rng(M * 7 + N * 3 + K + 10 * a_mn + b_mn)
    A = synth.round_bf16(r.standard_normal((M, K)))
    B = synth.round_bf16(r.standard_normal((N, K)))
    Ad = _bf16_dev(A.T, _ru8(M)) if a_mn else _bf16_dev(A, _ru8(K))
    lda = _ru8(M) if a_mn else _ru8(K)
    Bd = _bf16_dev(B.T, _ru8(N)) if b_mn else _bf16_dev(B, _ru8(K))
    ldb = _ru8(N) if b_mn else _ru8(K)
    bias = r.standard_normal(N).astype(np.float32)
    zin = r.standard_normal((M, N)).astype(np.float32)
    biasd = torch.as_tensor(bias).cuda()
    zind = torch.as_tensor(zin).cuda()
    D = A @ B.T
    bound = K * 2.0 ** -23 * (np.abs(A) @ np.abs(B).T) + 1e-30
    tctx = tdk.Context(0, testing=True)  # the raw GEMM entry is in the test build only
    L = tctx.L
    for mode in range(4):
        outf = torch.full((M, N), float("nan"), dtype=torch.float32, device="cuda")
        outb = torch.full((M, _ru8(N)), float("nan"), dtype=torch.bfloat16, device="cuda")
        rc = L.tdk_test_gemm_bf16(tctx.handle, M, N, K, Ad.data_ptr(), lda, a_mn, Bd.data_ptr(), ldb, b_mn, mode,
                                  biasd.data_ptr(), zind.data_ptr(), N, outf.data_ptr(), N, outb.data_ptr(), _ru8(N))
        assert rc == 0
        torch.cuda.synchronize()
        f = outf.cpu().double().numpy()
        bo = outb.float().cpu().double().numpy()[:, :N]
        if mode == 0:
            assert np.all(np.abs(f - D) <= bound)
        elif mode == 2:
            assert np.all(np.abs(f - (D + bias)) <= bound + 1e-6 * np.abs(bias))
        elif mode == 1:
            Z = D + bias
            assert np.all(np.abs(f - Z) <= bound + 1e-6 * np.abs(bias))
            ref = omlp.gelu(f)  # the kernel rounds gelu of its own pre-activation
            assert np.all(np.abs(bo - ref) <= 2.0 ** -7 * np.abs(ref) + 1e-6)
        else:
            ref = D * omlp.gelu_grad(zin)
            assert np.all(np.abs(bo - ref) <= 2.0 ** -7 * np.abs(ref) + bound * 2 + 1e-6)
    assert tctx.sync_status() == 0
    tctx.close()


def _odeco_cores(batch, Rt, N, seed, noise=1e-3):
    """Cores with well-separated spectra in every unfolding: sum_r w_r q1_r o
    q2_r o q3_r with orthogonal Q_n and distinct weights, plus small noise."""
    r = np.random.default_rng(seed)
    out = []
    for _ in range(batch):
        Qs = [np.linalg.qr(r.standard_normal((Rt, Rt)))[0] for _ in range(N)]
        w = np.linspace(2.0, 0.3, Rt) * (1.0 + 0.05 * r.random(Rt))
        G = oracle.cp_full(w, Qs) + noise * r.standard_normal((Rt,) * N)
        out.append(G)
    return np.array(out)


def _problem(batch, N, Rt, seed):
    r = np.random.default_rng(seed + 1)
    G = _odeco_cores(batch, Rt, N, seed)
    cs = r.standard_normal((batch, N, Rt)) * 3.0
    R = r.integers(2, Rt + 1, size=batch).astype(np.int32)
    Bs = r.standard_normal((batch, N, Rt, Rt))
    return G, cs, R, Bs


def _dev_batch(G, cs, R, Bs):
    import torch

    b = G.shape[0]
    return (torch.as_tensor(G.reshape(b, -1), dtype=torch.float32).cuda(), torch.as_tensor(cs).cuda(),
            torch.as_tensor(R).cuda(), torch.as_tensor(Bs).cuda())


def test_canonicalisation_matches_oracle(tdk, ctx):
    N, Rt, hidden, batch = 3, 6, 32, 9
    G, cs, R, Bs = _problem(batch, N, Rt, 21)
    m = tdk.Mlp(ctx, N, Rt, hidden, max_batch=16)
    m.set_params(synth.mlp_init_params(N, Rt, hidden, 1))
    Gd, csd, Rd, Bd = _dev_batch(G, cs, R, Bs)
    m.train_step(Gd, csd, Rd, Bd, alpha=0.5, update=False)
    S = m.get(tdk.MLP_CANON_CORE).reshape((batch,) + (Rt,) * N)
    V = m.get(tdk.MLP_ROTATIONS).reshape(batch, N, Rt, Rt)
    for s in range(batch):
        So, Vo, _ = omlp.canonicalise(G[s].astype(np.float32).astype(np.float64), cs[s])
        assert np.abs(S[s] - So).max() < 1e-4, s
        for n in range(N):
            assert np.abs(V[s, n] - Vo[n]).max() < 1e-4, (s, n)
    m.close()


@pytest.mark.parametrize("batch", [37, 150])
def test_loss_and_gradients_match_oracle(tdk, ctx, batch):
    N, Rt, hidden = 3, 6, 64
    alpha = 0.5
    G, cs, R, Bs = _problem(batch, N, Rt, 5 + batch)
    theta = synth.mlp_init_params(N, Rt, hidden, 2)
    m = tdk.Mlp(ctx, N, Rt, hidden, max_batch=256)
    m.set_params(theta)
    Gd, csd, Rd, Bd = _dev_batch(G, cs, R, Bs)
    import torch

    lam = np.random.default_rng(batch).uniform(0.5, 2.0, (batch, Rt))
    loss = m.train_step(Gd, csd, Rd, Bd, alpha=alpha, update=False, lam=torch.as_tensor(lam).cuda())
    g = m.get(tdk.MLP_GRADS).astype(np.float64)
    O = m.get(tdk.MLP_OUTPUT).reshape(batch, -1)
    # oracle from the same FP32 cores
    G32 = G.astype(np.float32).astype(np.float64)
    Ss, Ts = [], []
    for s in range(batch):
        S, V, nrm = omlp.canonicalise(G32[s], cs[s])
        Ss.append(S)
        Bw = [Bs[s, n][:, :R[s]] * (lam[s, :R[s]] if n == N - 1 else 1.0) for n in range(N)]
        Ts.append(omlp.canonical_target(Bw, V, nrm))
    Ss = np.array(Ss)
    X = omlp.network_input(Ss)
    Lo, go, Oo = omlp.loss_grad(theta.astype(np.float64), X, Ss, R, N, Rt, hidden, T=Ts, alpha=alpha, bf16=True)
    assert np.linalg.norm(O - Oo) <= 2e-3 * np.linalg.norm(Oo)
    assert abs(loss - Lo) <= 2e-3 * abs(Lo)
    sizes = omlp.param_sizes(N, Rt, hidden)
    o = 0
    for k, sz in enumerate(sizes):
        gg, gr = g[o:o + sz], go[o:o + sz]
        assert np.linalg.norm(gg - gr) <= 1e-2 * np.linalg.norm(gr) + 1e-12, (k, np.linalg.norm(gg - gr),
                                                                             np.linalg.norm(gr))
        o += sz
    m.close()


def test_adam_step_matches_oracle(tdk, ctx):
    N, Rt, hidden, batch = 3, 6, 32, 20
    G, cs, R, Bs = _problem(batch, N, Rt, 31)
    theta = synth.mlp_init_params(N, Rt, hidden, 3)
    m = tdk.Mlp(ctx, N, Rt, hidden, max_batch=32)
    m.set_params(theta)
    Gd, csd, Rd, Bd = _dev_batch(G, cs, R, Bs)
    m.train_step(Gd, csd, Rd, None, lr=1e-3, update=False)
    g = m.get(tdk.MLP_GRADS).astype(np.float64)
    m.train_step(Gd, csd, Rd, None, lr=1e-3, update=True)  # same batch: same gradient, then the step
    th = m.get(tdk.MLP_PARAMS).astype(np.float64)
    ref, _, _ = omlp.adam_step(theta.astype(np.float64), np.zeros_like(g), np.zeros_like(g), g, 1, 1e-3)
    assert np.abs(th - ref).max() <= 1e-6 * max(1.0, np.abs(ref).max())
    m.close()


def test_adam_step_with_gradient_clipping_matches_oracle(tdk, ctx):
    """clip > 0: the Adam step takes the gradient scaled to the cap
    (oracle.mlp.clip_grad); the stored gradient stays unscaled.  Two steps,
    since the first Adam step is nearly invariant to the gradient's scale."""
    N, Rt, hidden, batch = 3, 6, 32, 20
    G, cs, R, Bs = _problem(batch, N, Rt, 33)
    theta = synth.mlp_init_params(N, Rt, hidden, 5)
    m = tdk.Mlp(ctx, N, Rt, hidden, max_batch=32)
    m.set_params(theta)
    Gd, csd, Rd, Bd = _dev_batch(G, cs, R, Bs)
    m.train_step(Gd, csd, Rd, None, lr=1e-3, update=True)          # step 1, unclipped
    g1 = m.get(tdk.MLP_GRADS).astype(np.float64)
    m.train_step(Gd, csd, Rd, None, lr=1e-3, update=False)         # the gradient at the new point
    g2 = m.get(tdk.MLP_GRADS).astype(np.float64)
    cap = 0.25 * float(np.linalg.norm(g2))
    m.train_step(Gd, csd, Rd, None, lr=1e-3, update=True, clip=cap)  # step 2, clipped
    assert np.array_equal(m.get(tdk.MLP_GRADS).astype(np.float64), g2)
    th = m.get(tdk.MLP_PARAMS).astype(np.float64)
    z = np.zeros_like(g1)
    t1, m1, v1 = omlp.adam_step(theta.astype(np.float64), z, z, g1, 1, 1e-3)
    ref, _, _ = omlp.adam_step(t1, m1, v1, omlp.clip_grad(g2, cap), 2, 1e-3)
    unclipped, _, _ = omlp.adam_step(t1, m1, v1, g2, 2, 1e-3)
    err = np.abs(th - ref).max()
    assert err <= 1e-6 * max(1.0, np.abs(ref).max())
    assert np.abs(unclipped - ref).max() > 100 * err   # the clipping is visible at this tolerance
    m.close()


def test_predict_init_matches_oracle(tdk, ctx):
    import torch

    N, Rt, hidden, R = 3, 6, 64, 4
    shape = (30, 28, 26)
    r = np.random.default_rng(41)
    # tensor of exact multilinear rank Rt whose core has separated spectra
    G0 = _odeco_cores(1, Rt, N, 42, noise=0.0)[0]
    As = [np.linalg.qr(r.standard_normal((I, Rt)))[0] for I in shape]
    Y = oracle.tucker_full(G0, As)
    W = synth.sketch_matrices(shape, Rt, 43)
    Yd = dev_tensor(Y, "f32")
    U, _ = tdk.tucker_sketch(ctx, Yd, dev_W(W), [Rt] * N, 0, "simt")
    Gd, _ = tdk.tucker_core(ctx, Yd, U, [Rt] * N, 0, "simt")
    theta = synth.mlp_init_params(N, Rt, hidden, 4)
    m = tdk.Mlp(ctx, N, Rt, hidden, max_batch=4)
    m.set_params(theta)
    B = m.predict_init(Gd, U, shape, [Rt] * N, 0, tdk.F32, R)
    torch.cuda.synchronize()
    Gh = host(Gd)
    cs = [host(u).sum(axis=0) for u in U]
    S, V, _ = omlp.canonicalise(Gh, cs)
    O, _ = omlp.forward(theta.astype(np.float64), omlp.network_input(S[None]), N, Rt, hidden, bf16=True)
    Bh = [O[0, n * Rt * Rt:(n + 1) * Rt * Rt].reshape(Rt, Rt)[:, :R] for n in range(N)]
    ref = omlp.decanonicalise(Bh, V)
    for n in range(N):
        got = host(B[n])
        assert got.shape == (Rt, R)
        assert np.linalg.norm(got - ref[n]) <= 2e-3 * np.linalg.norm(ref[n])
    m.close()


def _method_problem(k, split, I, Rt, rmin):
    """Tensor k of the learned-initialiser workload at I^3, sketch width Rt."""
    import torch

    w = synth.learned_init_workload(k, split, (I,) * 3, Rt, rmin)
    Y, _ = synth.device_tensor(w, device="cuda")
    W = synth.sketch_matrices(w.shape, w.Rt, w.seed)
    Wd = [[None if x is None else torch.as_tensor(x, device="cuda") for x in row] for row in W]
    B0 = [torch.as_tensor(b, device="cuda") for b in synth.init_factors(w.Rt, w.als_R, w.seed)]
    return w, Y, Wd, B0, w.als_R


def test_learned_start_needs_fewer_sweeps(tdk, ctx):
    """Train the initialiser on cores and converged factors that the method
    generates, then compare ALS sweeps to convergence on held-out tensors from
    the random start, the HOSVD start and the learned start.  Asserted: the
    trained network beats the random start in median sweeps at an equal final
    fit.  The HOSVD start is measured beside it (on this workload it stays the
    fastest start; the comparison is reported, not asserted)."""
    from paper_1412_1885_gb300 import learned_init as li

    I, Rt, hidden, ntrain, ntest = 24, 8, 1024, 4096, 96
    m = tdk.Mlp(ctx, 3, Rt, hidden, max_batch=128)
    m.set_params(synth.mlp_init_params(3, Rt, hidden, 0, hosvd_start=True, out_scale=0.1))
    items = []
    for k in range(ntrain):
        w, Y, Wd, B0, R = _method_problem(k, 1, I, Rt, 3)
        items.append(li.method_sample(ctx, m, Y, Wd, [Rt] * 3, 0, R, B0, prec="simt", init="hosvd", max_sweeps=300))
    data = li.stack(items)
    assert data.G.shape[0] > 0.7 * ntrain
    hist = li.train(m, data, epochs=40, batch=128, lr=1e-3, alpha=0.5)
    assert hist[-1] < 0.5 * hist[0]
    sw = {"random": [], "hosvd": [], "learned": []}
    fit = {"random": [], "hosvd": [], "learned": []}
    for k in range(ntest):
        w, Y, Wd, B0, R = _method_problem(k, 2, I, Rt, 3)
        U, _ = tdk.tucker_sketch(ctx, Y, Wd, [Rt] * 3, 0, "simt")
        G, nrm = tdk.tucker_core(ctx, Y, U, [Rt] * 3, 0, "simt")
        runs = {"random": dict(B0=B0), "hosvd": dict(init="hosvd"),
                "learned": dict(B0=m.predict_init(G, U, w.shape, [Rt] * 3, 0, tdk.F32, R))}
        for name, kw in runs.items():
            o = tdk.ffcp_als(ctx, G, U, w.shape, [Rt] * 3, 0, tdk.F32, R, 1000, 1e-7, normY2=nrm, **kw)
            sw[name].append(o["sweeps"])
            fit[name].append(o["fit_Y"])
    med = {k: float(np.median(v)) for k, v in sw.items()}
    mean_fit = {k: float(np.mean(v)) for k, v in fit.items()}
    print("median sweeps", med, "mean final fit_Y", mean_fit)
    assert med["learned"] < med["random"], med
    # the same final fit: the learned start does not land in worse optima on average
    assert mean_fit["learned"] >= mean_fit["random"] - 2e-3, mean_fit
    m.close()


def test_layers_and_gradients_elementwise_at_full_width(tdk, ctx):
    """The workload's network (20^3 cores: 8000 -> 1024 -> 1024 -> 1200) on a
    batch of 64, every stored quantity and every gradient entry checked
    against the oracle's step fed with the kernels' own inputs of that step
    (the stored BF16 activations and deltas, exact values), so that each
    bound is the arithmetic of one step:
      FP32 products of BF16 values: |error| <= K 2^-23 sum |a b| (K terms);
      a BF16 store: one unit in the last place (2^-8 to 2^-7 relative), where
      the FP32 and FP64 values straddle a rounding boundary;
      dL/dO from the Gram identities in FP32: one BF16 unit plus 1e-4 of the
      sample's largest entry.
    Biases are random so that the bias terms are exercised."""
    import torch

    N, Rt, hidden, batch, alpha = 3, 20, 1024, 64, 0.5
    G, cs, R, Bs = _problem(batch, N, Rt, 77)
    theta = synth.mlp_init_params(N, Rt, hidden, 5).astype(np.float64)
    sizes = omlp.param_sizes(N, Rt, hidden)
    offs = np.concatenate([[0], np.cumsum(sizes)])
    r = np.random.default_rng(6)
    for k in (1, 3, 5):  # b1, b2, b3
        theta[offs[k]:offs[k + 1]] = 0.1 * r.standard_normal(sizes[k])
    theta = theta.astype(np.float32)
    m = tdk.Mlp(ctx, N, Rt, hidden, max_batch=batch)
    m.set_params(theta)
    Gd, csd, Rd, Bd = _dev_batch(G, cs, R, Bs)
    lam = r.uniform(0.5, 2.0, (batch, Rt))
    m.train_step(Gd, csd, Rd, Bd, alpha=alpha, update=False, lam=torch.as_tensor(lam).cuda())
    get = lambda what, cols: m.get(what).astype(np.float64).reshape(batch, cols)  # noqa: E731
    din, dout = Rt ** N, N * Rt * Rt
    X, Z1, H1 = get(tdk.MLP_INPUT, din), get(tdk.MLP_Z1, hidden), get(tdk.MLP_H1, hidden)
    Z2, H2, O = get(tdk.MLP_Z2, hidden), get(tdk.MLP_H2, hidden), get(tdk.MLP_OUTPUT, dout)
    dO, dZ2, dZ1 = get(tdk.MLP_DO, dout), get(tdk.MLP_DZ2, hidden), get(tdk.MLP_DZ1, hidden)
    S = m.get(tdk.MLP_CANON_CORE).astype(np.float64).reshape((batch,) + (Rt,) * N)
    V = m.get(tdk.MLP_ROTATIONS).astype(np.float64).reshape(batch, N, Rt, Rt)
    g = m.get(tdk.MLP_GRADS).astype(np.float64)
    W1, b1, W2, b2, W3, b3 = omlp.unpack(theta.astype(np.float64), N, Rt, hidden)
    q = synth.round_bf16
    u23 = 2.0 ** -23

    # the network input is the BF16 value of sqrt(Rt^N) vec S (scaled in FP32)
    xin = omlp.network_input(S)
    assert np.all(np.abs(X - q(xin)) <= bf16_ulp(np.maximum(np.abs(X), np.abs(xin))))

    def check_linear(Hin, Wt, b, Zout, name):
        ref = omlp.linear(Hin, Wt, b)
        bound = Hin.shape[1] * u23 * (np.abs(Hin) @ np.abs(q(Wt)).T + np.abs(b)) + 1e-30
        err = np.abs(Zout - ref)
        assert np.all(err <= bound), (name, float((err / bound).max()))

    def check_store(got, ref, name, extra=0.0):
        err = np.abs(got - ref)
        bound = bf16_ulp(np.maximum(np.abs(ref), np.abs(got))) + extra + 1e-30
        assert np.all(err <= bound), (name, float((err / bound).max()))

    check_linear(X, W1, b1, Z1, "Z1")
    check_store(H1, omlp.activation(Z1), "H1")
    check_linear(H1, W2, b2, Z2, "Z2")
    check_store(H2, omlp.activation(Z2), "H2")
    check_linear(H2, W3, b3, O, "O")
    # dL/dO from the kernel's O, S and target (with the kernel's rotations)
    G32 = G.astype(np.float32).astype(np.float64)
    Ts = []
    for s in range(batch):
        nrm = float(np.sqrt(np.sum(G32[s] ** 2)))
        Bw = [Bs[s, n][:, :R[s]] * (lam[s, :R[s]] if n == N - 1 else 1.0) for n in range(N)]
        Ts.append(omlp.canonical_target(Bw, [V[s, n] for n in range(N)], nrm))
    dOo = omlp.dloss_dO(O, S, R, Ts, alpha)
    check_store(dO, dOo, "dO", extra=1e-4 * np.abs(dOo).max(axis=1, keepdims=True))
    # deltas from the kernel's own upstream delta and pre-activation
    for got, dn, Wt, Z, K, name in ((dZ2, dO, W3, Z2, dout, "dZ2"), (dZ1, dZ2, W2, Z1, hidden, "dZ1")):
        ref = omlp.delta(dn, Wt, Z)
        acc = 2 * K * u23 * (np.abs(dn) @ np.abs(q(Wt))) * np.abs(omlp.gelu_grad(Z))
        check_store(got, ref, name, extra=acc)
    # weight and bias gradients: batch sums of exact BF16 products
    for k, (D, Hin) in zip((4, 2, 0), ((dO, H2), (dZ2, H1), (dZ1, X))):
        gw = g[offs[k]:offs[k + 1]].reshape(D.shape[1], Hin.shape[1])
        bound = batch * u23 * (np.abs(D).T @ np.abs(Hin)) + 1e-30
        assert np.all(np.abs(gw - D.T @ Hin) <= bound), k
        gb = g[offs[k + 1]:offs[k + 2]]
        assert np.all(np.abs(gb - D.sum(axis=0)) <= batch * u23 * np.abs(D).sum(axis=0) + 1e-30), k + 1
    # and the whole chain against the oracle run from the kernel's input
    Lo, go, Oo = omlp.loss_grad(theta.astype(np.float64), X, S, R, N, Rt, hidden, T=Ts, alpha=alpha, bf16=True)
    assert np.linalg.norm(O - Oo) <= 2e-3 * np.linalg.norm(Oo)
    for k in range(6):
        a, b = g[offs[k]:offs[k + 1]], go[offs[k]:offs[k + 1]]
        assert np.linalg.norm(a - b) <= 2e-2 * np.linalg.norm(b) + 1e-12, k
    m.close()
