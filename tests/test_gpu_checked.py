"""The checked build (libtdk_test.so, -DTDK_CHECKED): every entry point on odd
and tiny shapes, tensor-core and CUDA-core forms, with the bounds checks of
the kernels' index computations armed.  A failed check skips the access and
raises TDK_STATUS_OOB (bit 512) in the status word, so each case asserts a
clean status, and results equal to the product library's up to rounding (the
checks can change how the compiler contracts multiply-adds)."""
import numpy as np
import pytest

import synth
from helpers import dev_tensor, dev_W, host, small_problem

pytestmark = pytest.mark.gpu

OOB = 512


@pytest.fixture(scope="module")
def tdk():
    import paper_1412_1885_gb300 as t
    from paper_1412_1885_gb300 import build

    build.build()
    return t


@pytest.fixture(scope="module")
def ctxs(tdk):
    chk, prod = tdk.Context(0, testing=True), tdk.Context(0)
    yield chk, prod
    chk.close()
    prod.close()


def test_a_failed_check_is_reported_and_the_access_skipped(tdk, ctxs):
    chk, _ = ctxs
    assert chk.L.tdk_test_checked_store(chk.handle, 3, 4) == 0
    assert chk.sync_status() == 0
    assert chk.L.tdk_test_checked_store(chk.handle, 4, 4) == 0   # one past the end: skipped
    assert chk.sync_status() & OOB
    assert chk.L.tdk_test_checked_store(chk.handle, -1, 4) == 0
    assert chk.sync_status() & OOB
    assert chk.sync_status() == 0   # read and cleared


CASES = [
    ("f64", "simt", (7, 5, 9), (2, 2, 3), 1),
    ("f32", "simt", (67, 45, 130), (4, 5, 3), 3),
    ("bf16", "simt", (9, 11, 7, 13), (2, 3, 2, 3), 2),
    ("bf16", "tc", (67, 45, 136), (4, 5, 3), 3),
    ("bf16", "tc", (300, 130, 72), (10, 12, 9), 6),
    ("f32", "tc", (33, 70, 64), (4, 4, 4), 3),
    ("bf16", "tc", (12, 10, 9, 16), (3, 4, 2, 5), 2),
]


@pytest.mark.parametrize("dtype,prec,shape,ranks,p", CASES)
def test_compression_paths_pass_the_bounds_checks(tdk, ctxs, dtype, prec, shape, ranks, p):
    chk, prod = ctxs
    Y, W, _ = small_problem(shape, ranks, p, seed=19, dtype=dtype)
    Yd, Wd = dev_tensor(Y, dtype), dev_W(W)
    out = {}
    for name, c in (("chk", chk), ("prod", prod)):
        U, _ = tdk.tucker_sketch(c, Yd, Wd, ranks, p, prec)
        G, nrm = tdk.tucker_core(c, Yd, U, ranks, p, prec)
        Us, Gs, _ = tdk.tucker_seq(c, Yd, Wd, ranks, p, prec)
        Rt = [r + p for r in ranks]
        U2 = [dev_tensor(u, "f64") for u in synth.random_factors(shape, Rt, 19)]
        tdk.tucker_refine(c, Yd, dev_W(synth.refine_matrices(Rt, 19, 0)), U2, ranks, p, prec=prec)
        assert c.sync_status() == 0, name
        out[name] = [host(u) for u in U] + [host(G)] + [host(u) for u in Us] + [host(Gs)] + [host(u) for u in U2]
    tol = 1e-11 if dtype == "f64" else 1e-4
    for a, b in zip(out["chk"], out["prod"]):
        assert np.allclose(a, b, rtol=tol, atol=tol * np.abs(b).max())


@pytest.mark.parametrize("dtype,core,R,nonneg,form", [
    ("f32", (6, 5, 7), 3, False, None),           # one CTA
    ("f64", (9, 8, 7, 6), 4, False, None),        # persistent grid, 4-way
    ("f32", (9, 8, 7, 6), 4, True, None),         # nonneg on the grid
    ("f32", (10, 9, 8), 3, True, "steps"),        # kernel-per-step form
    ("f64", (10, 9, 8), 3, False, "steps"),
])
def test_ffcp_forms_pass_the_bounds_checks(tdk, ctxs, dtype, core, R, nonneg, form):
    chk, prod = ctxs
    shape = tuple(2 * c + 3 for c in core)
    ranks, p = [c - 1 for c in core], 1
    rng = np.random.default_rng(5)
    G = rng.standard_normal(core)
    U = [np.linalg.qr(rng.standard_normal((i, c)))[0] for i, c in zip(shape, core)]
    Gd, Ud = dev_tensor(G, dtype), [dev_tensor(u, "f64") for u in U]
    kw = dict(max_sweeps=12, tol=0.0, form=form)
    if nonneg:
        kw["A0"] = [dev_tensor(np.abs(rng.standard_normal((i, R))), "f64") for i in shape]
        kw["nonneg"] = True
    else:
        kw["B0"] = [dev_tensor(rng.standard_normal((c, R)), "f64") for c in core]
    res = {}
    for name, c in (("chk", chk), ("prod", prod)):
        o = tdk.ffcp_als(c, Gd, Ud, shape, ranks, p, 0 if dtype == "f64" else 1, R, **kw)
        assert c.sync_status() == 0, name
        res[name] = [host(a) for a in o["A"]]
    tol = 1e-9 if dtype == "f64" else 1e-3
    for a, b in zip(res["chk"], res["prod"]):
        assert np.allclose(a, b, rtol=tol, atol=tol * np.abs(b).max())
