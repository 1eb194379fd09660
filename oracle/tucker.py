"""Oracle: randomized Tucker compression (Sec. IV-A, Alg. 2) in FP64.

TEST INFRASTRUCTURE ONLY (see the package docstring): only tests, smoke()
and bench.py's CPU legs may use it.

The method computes, for every mode n from the ORIGINAL tensor Y,
  Z_n = Y_(n) Omega_n,   Omega_n = KRP_{k != n} W_k^(n)          (RRF step 2)
  U_n = orthonormal basis of range(Z_n) by Householder QR        (RRF step 3)
  G   = Y x_1 U_1^T x_2 ... x_N U_N^T                            (Alg. 2, TTM)
i.e. the range-finder sketch of every mode taken in one pass over Y with a
Khatri-Rao structured Gaussian test matrix, then the Tucker core (Eq. 1).

The forms the paper prints are here too: the range finder with a dense
Gaussian Omega (`rand_tucker_dense`), Alg. 2's sequential sketch on the
shrinking tensor (`rand_tucker_seq`, and `rand_tucker_seq_krp` with
Khatri-Rao test matrices), the Gram-based basis of Eq. 23 (`evd_orth`), the
sub-tensor grid of Sec. IV-B (`rand_tucker_grid`) and RandTucker2i (Alg. 3).
"""
from __future__ import annotations

import numpy as np


def norm2(Y) -> float:
    """||Y||_F^2 (used by the fit, Sec. III-B).  Pinned: the explicit sum of
    squares in the sketch's brute-force test."""
    Y = np.asarray(Y, dtype=np.float64)
    return float(np.sum(Y * Y))


def unfold(Y: np.ndarray, n: int) -> np.ndarray:
    """Mode-n matricization Y_(n) (Table I): rows i_n, columns the other
    indices in row-major order.  Pinned by brute force in tests."""
    return np.moveaxis(np.asarray(Y, dtype=np.float64), n, 0).reshape(Y.shape[n], -1)


def fold(M: np.ndarray, n: int, shape) -> np.ndarray:
    """Inverse of unfold for a tensor of the given shape.  Pinned: the
    round trip of the index-loop unfolding test, and through the TTM pins."""
    shape = list(shape)
    lead = [shape[n]] + shape[:n] + shape[n + 1:]
    return np.moveaxis(M.reshape(lead), 0, n)


def khatri_rao(mats) -> np.ndarray:
    """Column-wise Kronecker product (Table I), first factor slowest.

    (A (.) B)[(i, j), r] = A[i, r] * B[j, r].  Pinned by the identity
    (A (.) B)^T (A (.) B) = A^T A * B^T B (Eq. 9) and by brute force.
    """
    mats = [np.asarray(m, dtype=np.float64) for m in mats]
    R = mats[0].shape[1]
    out = mats[0]
    for m in mats[1:]:
        out = (out[:, None, :] * m[None, :, :]).reshape(-1, R)
    return out


def sketch(Y: np.ndarray, W) -> tuple[list, float]:
    """All-mode range-finder sketch (Sec. IV-A step 2; Alg. 2, the sketch of each mode).

    Z_n = Y_(n) Omega_n with Omega_n = KRP_{k != n} W[n][k] formed explicitly,
    for every n from the same (original) Y; also returns ||Y||^2.
    Pinned: brute-force loops, rank-one closed form (tests).
    """
    Y = np.asarray(Y, dtype=np.float64)
    N = Y.ndim
    Z = []
    for n in range(N):
        Omega = khatri_rao([W[n][k] for k in range(N) if k != n])
        Z.append(unfold(Y, n) @ Omega)
    return Z, norm2(Y)


def sketch_row(slab: np.ndarray, n: int, W, chunk: int = 32) -> np.ndarray:
    """One row Z_n[i, :] from the slab Y[..., i_n = i, ...] (shape: the other
    modes in order).  Same definition as `sketch`; Omega_n is formed a block of
    its rows at a time (the first remaining index in chunks) so that rows of
    full-size problems fit in host memory.  Pinned: equals the rows of the
    brute-force-pinned `sketch`.
    """
    slab = np.asarray(slab, dtype=np.float64)
    N = slab.ndim + 1
    facs = [W[n][k] for k in range(N) if k != n]
    out = np.zeros(facs[0].shape[1])
    rest = facs[1:]
    for a in range(0, slab.shape[0], chunk):
        b = min(slab.shape[0], a + chunk)
        Om = khatri_rao([facs[0][a:b]] + rest)
        out += slab[a:b].reshape(-1) @ Om
    return out


def householder_qr(Z: np.ndarray):
    """Thin QR by Householder reflections (Sec. IV-A step 3, which names QR as one way).

    Returns Q (m x k, orthonormal columns) and R (k x k, upper triangular)
    with Z = Q R and diag(R) >= 0 (sign convention that makes Q unique for
    full-rank Z).  Pinned: Q^T Q = I, QR = Z, triangularity, and agreement
    with LAPACK's QR after the same sign fix (tests).
    """
    A = np.array(Z, dtype=np.float64)
    m, k = A.shape
    if k > m:
        raise ValueError("QR needs rows >= columns")
    vs = []
    for j in range(k):
        x = A[j:, j]
        nx = np.linalg.norm(x)
        if nx == 0.0:
            vs.append(None)
            continue
        alpha = -nx if x[0] >= 0 else nx
        v = x.copy()
        v[0] -= alpha
        nv = np.linalg.norm(v)
        if nv == 0.0:
            vs.append(None)
            continue
        v /= nv
        A[j:, j:] -= 2.0 * np.outer(v, v @ A[j:, j:])
        vs.append(v)
    R = np.triu(A[:k, :k])
    Q = np.zeros((m, k))
    Q[:k, :k] = np.eye(k)
    for j in reversed(range(k)):
        v = vs[j]
        if v is not None:
            Q[j:, :] -= 2.0 * np.outer(v, v @ Q[j:, :])
    s = np.where(np.diag(R) < 0, -1.0, 1.0)
    return Q * s[None, :], R * s[:, None]


def ttm(Y: np.ndarray, U: np.ndarray, n: int) -> np.ndarray:
    """Y x_n U^T (Alg. 2, the mode-n projection step): contracts mode n of Y with the
    columns of U, (Y x_n U^T)_(n) = U^T Y_(n).  Pinned: exact Tucker tensors."""
    Y = np.asarray(Y, dtype=np.float64)
    shape = list(Y.shape)
    shape[n] = U.shape[1]
    return fold(np.asarray(U, dtype=np.float64).T @ unfold(Y, n), n, shape)


def tucker_core(Y: np.ndarray, Us) -> np.ndarray:
    """G = Y x_1 U_1^T x_2 ... x_N U_N^T (Alg. 2, final core; Eq. 1).
    Pinned: recovers the core of an exact Tucker tensor in any mode order;
    Pythagoras ||Y - [[G; U]]||^2 = ||Y||^2 - ||G||^2."""
    G = np.asarray(Y, dtype=np.float64)
    for n, U in enumerate(Us):
        G = ttm(G, U, n)
    return G


def tucker_full(G: np.ndarray, Us) -> np.ndarray:
    """[[G; U_1, ..., U_N]] = G x_1 U_1 ... x_N U_N (Eq. 1).  Pinned with
    `tucker_core` (exact Tucker tensors, Pythagoras)."""
    X = np.asarray(G, dtype=np.float64)
    for n, U in enumerate(Us):
        shape = list(X.shape)
        shape[n] = U.shape[0]
        X = fold(np.asarray(U, dtype=np.float64) @ unfold(X, n), n, shape)
    return X


def hosvd_factors(Y: np.ndarray, ranks):
    """HOSVD factors: the leading R_n left singular vectors of every Y_(n)
    (Sec. II).  The full-tensor SVD is exactly the cost the randomized method
    avoids; the oracle keeps it as the deterministic reference compression.
    Pinned: exact recovery of exact multilinear-rank tensors, and the
    Eckart-Young residual against the eigenvalues of Y_(n) Y_(n)^T."""
    out = []
    for n, Rn in enumerate(ranks):
        Un, _, _ = np.linalg.svd(unfold(Y, n), full_matrices=False)
        out.append(Un[:, :Rn])
    return out


def rand_tucker(Y: np.ndarray, W) -> dict:
    """All-mode randomized Tucker: sketch every mode from the original Y,
    orthonormalise each sketch by Householder QR, then project to the core.

    Differs from the paper's Alg. 2 in one respect: Alg. 2 sketches mode n of
    the tensor already projected on modes < n; here every Z_n comes from the
    original Y (one pass for all modes), with Omega_n a Khatri-Rao product of
    small Gaussians instead of a dense Gaussian matrix.
    Pinned: exact recovery of exact multilinear-rank tensors (independent and
    shared sketch families); its accuracy against the printed forms is
    measured in the tests.
    """
    Z, nY2 = sketch(Y, W)
    QR = [householder_qr(z) for z in Z]
    U = [q for q, _ in QR]
    G = tucker_core(Y, U)
    return {"Z": Z, "U": U, "R": [r for _, r in QR], "G": G, "normY2": nY2}


def evd_orth(Z: np.ndarray, slabs: int = 1) -> np.ndarray:
    """Orthonormal basis of range(Z) by the Gram route of Sec. IV-B (Eq. 23):
    the Gram sum_s Z_s^T Z_s over `slabs` row blocks Z_s of Z has the
    eigendecomposition V Sigma V^T (eigenvalues decreasing), and every block
    of the basis is U_s = Z_s V Sigma^{-1/2}.  Eq. 23 divides by Sigma^{1/2},
    so Z must have full column rank (ValueError otherwise).  Pinned: U^T U = I,
    the projector U U^T equals that of the Householder basis, and the slab
    count changes only rounding."""
    Z = np.asarray(Z, dtype=np.float64)
    blocks = np.array_split(Z, slabs, axis=0)
    C = np.zeros((Z.shape[1], Z.shape[1]))
    for Zs in blocks:
        C += Zs.T @ Zs
    w, V = np.linalg.eigh(C)
    order = np.argsort(-w, kind="stable")
    w, V = w[order], V[:, order]
    if not w[-1] > Z.shape[1] * np.finfo(np.float64).eps * w[0]:
        raise ValueError("the Gram route needs Z of full column rank")
    return np.vstack([Zs @ (V / np.sqrt(w)[None, :]) for Zs in blocks])


def rand_tucker_dense(Y: np.ndarray, Omegas) -> dict:
    """All-mode randomized Tucker with the dense Gaussian test matrices of the
    range finder as printed (Sec. IV-A, step 1): Z_n = Y_(n) Omega_n with
    Omega_n of (prod_{k != n} I_k) x Rt_n given in full, every Z_n from the
    original Y, Householder bases, then the core.  The method's own sketch
    replaces Omega_n by a Khatri-Rao product; this form measures what that
    costs.  Pinned: exact recovery of exact multilinear-rank tensors."""
    Y = np.asarray(Y, dtype=np.float64)
    U = [householder_qr(unfold(Y, n) @ np.asarray(Omegas[n], dtype=np.float64))[0] for n in range(Y.ndim)]
    return {"U": U, "G": tucker_core(Y, U)}


def rand_tucker_seq(Y: np.ndarray, Omegas, orth: str = "qr") -> dict:
    """Alg. 2 as printed: for n = 1..N in order, Z_n = Y_(n) Omega_n with a
    dense Gaussian Omega_n, U_n an orthonormal basis of Z_n, then Y <- Y x_n
    U_n^T (mode n shrinks to Rt_n before mode n + 1 is sketched); the last Y
    is the core.  Omega_n therefore has prod_{k<n} Rt_k prod_{k>n} I_k rows.
    orth "qr" takes the Householder basis (step 3 names QR as one choice), "evd" the Gram
    route of Eq. 23.  Pinned: exact recovery, and the core equals the TTM
    chain of the original Y with the same factors."""
    X = np.asarray(Y, dtype=np.float64)
    U = []
    for n in range(X.ndim):
        Z = unfold(X, n) @ np.asarray(Omegas[n], dtype=np.float64)
        Un = householder_qr(Z)[0] if orth == "qr" else evd_orth(Z)
        U.append(Un)
        X = ttm(X, Un, n)
    return {"U": U, "G": X}


def seq_test_matrices(shape, W) -> list:
    """Khatri-Rao test matrices for Alg. 2's sequential sketch, drawn like
    the one-pass sketch's: Omega_n = KRP_{k != n} W[n][k][:d_k], with d_k the
    size of mode k at the time mode n is sketched (Rt_k for k < n, the modes
    already shrunk; I_k for k > n).  W[n][k] has at least d_k rows; only its
    first d_k rows enter.  Pinned: the mixed-product identity of the
    sequential sketch (tests)."""
    N = len(shape)
    Rt = [np.asarray(W[n][(n + 1) % N]).shape[1] for n in range(N)]
    out = []
    for n in range(N):
        rows = [Rt[k] if k < n else shape[k] for k in range(N)]
        out.append(khatri_rao([np.asarray(W[n][k], dtype=np.float64)[:rows[k]] for k in range(N) if k != n]))
    return out


def rand_tucker_seq_krp(Y: np.ndarray, W, orth: str = "qr") -> dict:
    """Alg. 2 (`rand_tucker_seq`) with the Khatri-Rao test matrices of
    `seq_test_matrices` in place of dense Gaussian ones; also returns
    ||Y||^2.  Pinned: exact recovery, and each Z_n equals the sketch of the
    original Y with the factors U_k W[n][k] for the shrunk modes (tests)."""
    Y = np.asarray(Y, dtype=np.float64)
    out = rand_tucker_seq(Y, seq_test_matrices(Y.shape, W), orth)
    out["normY2"] = norm2(Y)
    return out


def grid_blocks(shape, grid):
    """Index ranges of the sub-tensor grid of Sec. IV-B (Eq. 19): mode n is
    cut into grid[n] contiguous, near-equal blocks.  Returns one list of index
    arrays per mode."""
    return [np.array_split(np.arange(I), S) for I, S in zip(shape, grid)]


def sketch_share(Ysub: np.ndarray, idx, W) -> list:
    """One sub-tensor's contribution to every sketch (Eq. 22): for mode n,
    Y^(s)_(n) Omega_k, with Omega_k the rows of Omega_n = KRP_{k != n}
    W[n][k] that belong to the sub-tensor's index ranges idx[k] (the
    Khatri-Rao product of the row blocks of the small factors).  It adds into
    rows idx[n] of Z_n; the sum over all sub-tensors is the full sketch."""
    Ysub = np.asarray(Ysub, dtype=np.float64)
    N = Ysub.ndim
    return [unfold(Ysub, n) @ khatri_rao([W[n][k][idx[k]] for k in range(N) if k != n]) for n in range(N)]


def core_share(Ysub: np.ndarray, idx, Us) -> np.ndarray:
    """One sub-tensor's share of the core: Y^(s) x_1 U_1[idx_1]^T ... x_N
    U_N[idx_N]^T, with U_n[idx_n] the row block of U_n on the sub-tensor's
    range; the core is the sum of the shares (Sec. IV-B, last step)."""
    return tucker_core(Ysub, [np.asarray(U, dtype=np.float64)[idx[n]] for n, U in enumerate(Us)])


def rand_tucker_grid(Y: np.ndarray, W, grid) -> dict:
    """The all-mode randomized Tucker of `rand_tucker` computed as Sec. IV-B
    lays it out over a grid of sub-tensors:
      Z_n rows of block s_n = sum over the other blocks of the shares (Eq. 22),
      U_n = the Gram basis of Eq. 23 from the row-block Grams of Z_n,
      G   = sum of the sub-tensors' core shares.
    The partial sums are reduced here; the paper's "broadcast" of them is read
    as that reduction.  Pinned: equals the one-block sketch and core."""
    Y = np.asarray(Y, dtype=np.float64)
    N = Y.ndim
    blocks = grid_blocks(Y.shape, grid)
    Rt = [W[n][(n + 1) % N].shape[1] for n in range(N)]
    Z = [np.zeros((Y.shape[n], Rt[n])) for n in range(N)]
    cells = list(np.ndindex(*grid))
    for cell in cells:
        idx = [blocks[n][cell[n]] for n in range(N)]
        sub = Y[np.ix_(*idx)]
        for n, part in enumerate(sketch_share(sub, idx, W)):
            Z[n][idx[n]] += part
    U = [evd_orth(Z[n], slabs=grid[n]) for n in range(N)]
    G = np.zeros(Rt)
    for cell in cells:
        idx = [blocks[n][cell[n]] for n in range(N)]
        G += core_share(Y[np.ix_(*idx)], idx, U)
    return {"Z": Z, "U": U, "G": G}


def refine_pass(Y: np.ndarray, Us, W) -> list:
    """One pass of the RandTucker2i loop (Alg. 3, the body repeated twice),
    modes in order, each using the factors already refined in this pass:
        X   = Y x_{p != n} U_p^T                  (Alg. 3 prints U_p; read U_p^T)
        Z_n = X_(n) Omega_n,  Omega_n = KRP_{k != n} W[n][k]   (W[n][k]: Rt_k x Rt_n)
        U_n = orth(Z_n)                            (Householder QR, diag(R) >= 0)
    Omega_n is drawn as a Khatri-Rao product of small Gaussians, as for the
    first sketch.  Returns the new factor list.  Pinned through
    `rand_tucker_2i`."""
    Y = np.asarray(Y, dtype=np.float64)
    N = Y.ndim
    Us = [np.asarray(u, dtype=np.float64) for u in Us]
    for n in range(N):
        X = Y
        for p in range(N):
            if p != n:
                X = ttm(X, Us[p], p)
        Z = unfold(X, n) @ khatri_rao([W[n][k] for k in range(N) if k != n])
        Us[n], _ = householder_qr(Z)
    return Us


def rand_tucker_2i(Y: np.ndarray, U_init, W_passes) -> dict:
    """RandTucker2i (Alg. 3): random starting factors, two refinement passes
    (`refine_pass` with the sketch matrices of each pass), then the core.
    Pinned: exact recovery of exact multilinear-rank tensors; on noisy
    tensors, HOSVD <= RandTucker2i < one randomized pass in error (Fig. 5)."""
    Us = [np.asarray(u, dtype=np.float64) for u in U_init]
    for W in W_passes:
        Us = refine_pass(Y, Us, W)
    G = tucker_core(Y, Us)
    return {"U": Us, "G": G, "normY2": float(np.sum(np.asarray(Y, dtype=np.float64) ** 2))}
