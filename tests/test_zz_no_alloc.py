"""The allocation-free sketch entry point (tucker_sketch_static) against the
allocating one (tucker_sketch, CUDA-core form) on the same seeded inputs, on
two calls in a row that share the static scratch array.  This file is
collected last and also passes alone in a fresh process."""
import numpy as np
import pytest

from helpers import TOL_SKETCH, dev_tensor, dev_W, host, sketch_abs_bound, small_problem

pytestmark = pytest.mark.gpu

CASES = [
    ((67, 45, 130), "f32"),       # 47 row tiles + tail, 4 column chunks + tail
    ((67, 45, 130), "f64"),
    ((33, 70, 64), "bf16"),
    ((9, 11, 7, 13), "f32"),      # 4-way, ragged
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


@pytest.mark.parametrize("shape,dtype", CASES)
def test_static_sketch_matches_allocating_sketch(tdk, ctx, shape, dtype):
    import torch

    ranks = [min(4, s - 3) for s in shape]
    p = 3
    Y, W, _ = small_problem(shape, ranks, p, seed=11, dtype=dtype)
    Yd, Wd = dev_tensor(Y, dtype), dev_W(W)
    _, Zref = tdk.tucker_sketch(ctx, Yd, Wd, ranks, p, "simt", want_Z=True)
    bnd = sketch_abs_bound(Y, W)
    tol = TOL_SKETCH[(dtype, "simt")]
    outs = []
    for _call in range(2):
        # outputs start as NaN so that an element the call does not write fails
        Z = [torch.full((shape[n], ranks[n] + p), float("nan"), dtype=torch.float64, device="cuda")
             for n in range(len(shape))]
        tdk.tucker_sketch_static(ctx, Yd, Wd, ranks, p, Z_out=Z)
        torch.cuda.synchronize()
        outs.append([host(z) for z in Z])
        for n in range(len(shape)):
            err = np.abs(outs[-1][n] - host(Zref[n]))
            assert np.all(err <= tol * bnd[n] + 1e-300), (n, float(np.nanmax(err / bnd[n])))
    # the two calls share the scratch array and the launch shape: identical sums
    for n in range(len(shape)):
        assert np.array_equal(outs[0][n], outs[1][n])
    assert ctx.sync_status() == 0


def test_static_sketch_allocates_nothing(tdk):
    """The property the entry point exists for.  On a fresh context the call
    leaves the context's workspace at zero bytes and torch's allocator
    untouched; and in the test build, with every workspace growth made to
    fail, the call still succeeds (the allocating sketch is refused)."""
    import torch

    shape, ranks, p = (67, 45, 130), [4, 4, 4], 3
    Y, W, _ = small_problem(shape, ranks, p, seed=12, dtype="f32")
    Yd, Wd = dev_tensor(Y, "f32"), dev_W(W)
    Z = [torch.empty((shape[n], ranks[n] + p), dtype=torch.float64, device="cuda") for n in range(3)]
    torch.cuda.synchronize()
    for testing in (False, True):
        c = tdk.Context(0, testing=testing)
        if testing:
            assert c.L.tdk_ctx_test_fail_alloc(c.handle, 0) == 0  # any growth now fails
            with pytest.raises(tdk.TdkError) as e:
                tdk.tucker_sketch(c, Yd, Wd, ranks, p, "simt")
            assert e.value.code == tdk.TDK_ENOMEM
        before = torch.cuda.memory_allocated()
        assert c.workspace_bytes() == 0
        for _call in range(2):
            tdk.tucker_sketch_static(c, Yd, Wd, ranks, p, Z_out=Z)
        assert c.sync_status() == 0
        assert c.workspace_bytes() == 0
        assert torch.cuda.memory_allocated() == before
        c.close()


def test_static_sketch_rejects_problems_beyond_the_array(tdk, ctx):
    import torch

    # packed FP64 sketch alone: 64 * (64 + 64 + 70000) * 8 B = 36 MB > 16 MiB
    shape, ranks, p = (64, 64, 70000), [62, 62, 62], 2
    Y = torch.zeros(shape, dtype=torch.bfloat16, device="cuda")
    W = [[None if k == n else torch.zeros((shape[k], ranks[n] + p), dtype=torch.float64, device="cuda")
          for k in range(3)] for n in range(3)]
    before = ctx.launch_count()
    with pytest.raises(tdk.TdkError) as e:
        tdk.tucker_sketch_static(ctx, Y, W, ranks, p)
    assert e.value.code == tdk.TDK_ESCRATCH
    assert "static scratch" in str(e.value)
    assert ctx.launch_count() == before
