"""Host logic of the seeded input generators (no GPU)."""
import numpy as np
import pytest

import synth


@pytest.mark.parametrize("Rt", [[7, 7, 7], [5, 7, 6, 7]])
def test_shared_sketch_family_structure(Rt):
    shape = tuple(10 + 3 * n for n in range(len(Rt)))
    N = len(shape)
    W = synth.sketch_matrices(shape, Rt, 4, shared=True)
    wmax = max(Rt)
    for n in range(N):
        assert W[n][n] is None
        for k in range(N):
            if k == n:
                continue
            assert W[n][k].shape == (shape[k], Rt[n])
            # every sketch uses the leading columns of the one matrix of mode k
            full = next(W[m][k] for m in range(N) if m != k and Rt[m] == wmax)
            assert np.array_equal(W[n][k], full[:, :Rt[n]])
            if Rt[n] == wmax:
                assert W[n][k] is full
    # the independent family draws a different matrix for every (n, k)
    Wi = synth.sketch_matrices(shape, Rt, 4)
    assert not np.array_equal(Wi[0][N - 1], Wi[1][N - 1][:, :Rt[0]])


def test_shared_sketch_values_are_bf16_gaussian():
    W = synth.sketch_matrices((4000, 3000, 2000), 60, 1, shared=True)
    x = W[0][1]
    assert np.array_equal(x, synth.round_bf16(x))
    assert abs(x.mean()) < 0.01 and abs(x.std() - 1.0) < 0.01


def test_device_sketch_keeps_shared_objects_as_one_tensor():
    W = synth.sketch_matrices((6, 7, 8), 4, 2, shared=True)
    Wd = synth.device_sketch(W, "cpu")
    assert Wd[0][2] is Wd[1][2] and Wd[0][1] is Wd[2][1] and Wd[1][0] is Wd[2][0]
    Wi = synth.device_sketch(synth.sketch_matrices((6, 7, 8), 4, 2), "cpu")
    assert Wi[0][2] is not Wi[1][2]
    for n in range(3):
        for k in range(3):
            if k != n:
                assert np.array_equal(Wd[n][k].numpy(), W[n][k])


def test_sparse_exponential_factors_zero_share_and_mean():
    A = synth.sparse_exponential_factors((200, 300), 10, 5, mean=10.0, zero_frac=0.1)
    for I, a in zip((200, 300), A):
        assert a.shape == (I, 10) and np.all(a >= 0.0)
        assert int(np.sum(a == 0.0)) == round(0.1 * I * 10)
        nz = a[a > 0.0]
        # exponential(10): mean 10, std 10; nz has >= 1800 draws
        assert abs(nz.mean() - 10.0) < 1.0
    B = synth.sparse_exponential_factors((200, 300), 10, 5, mean=10.0, zero_frac=0.1)
    assert all(np.array_equal(a, b) for a, b in zip(A, B))
