"""Failure detection without a GPU fault: a device wait that runs out of time
(a barrier that nothing completes) must come back as a status bit and leave
the context usable; a workspace allocation failure and an ALS time limit must
come back as error codes.  The first two use the test build of the library
(libtdk_test.so), which alone carries the hooks that stage the failures."""
import numpy as np
import pytest

import oracle
import synth
from helpers import dev_tensor, dev_W, host, small_problem

pytestmark = pytest.mark.gpu

TDK_STATUS_TIMEOUT = 256


@pytest.fixture(scope="module")
def tdk():
    import paper_1412_1885_gb300 as t
    from paper_1412_1885_gb300 import build

    build.build()
    return t


def _small_sketch(tdk, ctx):
    shape, ranks, p = (30, 28, 26), (3, 3, 3), 2
    Y, W, _ = small_problem(shape, ranks, p, seed=4, dtype="f32")
    U, _ = tdk.tucker_sketch(ctx, dev_tensor(Y, "f32"), dev_W(W), ranks, p, "simt")
    return Y, W, U


def test_bounded_wait_times_out_into_the_status_word(tdk):
    ctx = tdk.Context(0, testing=True)
    assert ctx.sync_status() == 0
    assert ctx.L.tdk_test_bounded_wait(ctx.handle, 2_000_000) == 0  # 2 ms
    assert ctx.sync_status() & TDK_STATUS_TIMEOUT
    assert ctx.sync_status() == 0  # read and cleared
    # the context and the device stay usable
    Y, W, U = _small_sketch(tdk, ctx)
    Un = host(U[0])
    assert np.abs(Un.T @ Un - np.eye(Un.shape[1])).max() < 1e-12
    assert ctx.sync_status() == 0
    ctx.close()


def test_workspace_allocation_failure_returns_enomem(tdk):
    ctx = tdk.Context(0, testing=True)
    assert ctx.L.tdk_ctx_test_fail_alloc(ctx.handle, 0) == 0  # the next growth fails
    with pytest.raises(tdk.TdkError) as e:
        _small_sketch(tdk, ctx)
    assert e.value.code == tdk.TDK_ENOMEM
    assert ctx.L.tdk_ctx_test_fail_alloc(ctx.handle, -1) == 0  # growth allowed again
    _small_sketch(tdk, ctx)
    assert ctx.sync_status() == 0
    ctx.close()


def test_als_time_limit_returns_timeout_with_an_iterate(tdk):
    ctx = tdk.Context(0)
    shape, ranks, p, R = (40, 36, 32), (5, 5, 5), 3, 4
    Y, W, _ = small_problem(shape, ranks, p, seed=5, dtype="f64", snr=20.0, R_cp=R)
    ref = oracle.rand_tucker(Y, W)
    B0 = [dev_tensor(b, "f64") for b in synth.init_factors([r + p for r in ranks], R, 1)]
    with pytest.raises(tdk.TdkError) as e:
        tdk.ffcp_als(ctx, dev_tensor(ref["G"], "f64"), [dev_tensor(u, "f64") for u in ref["U"]], shape, ranks, p,
                     0, R, max_sweeps=100000, tol=0.0, B0=B0, timeout_s=1e-3)
    assert e.value.code == tdk.TDK_ETIMEOUT
    assert ctx.sync_status() == 0
    ctx.close()
