"""Oracle: FFCP, i.e. CP-ALS on the Tucker core, lifted back (Sec. III-B, Alg. 1).

TEST INFRASTRUCTURE ONLY (see the package docstring).

With orthonormal U_n, FFCP on Y~ = [[G; U]] is equivalent to CP of the core
(Eq. 17): for every mode n
  H_n = G_(n) [KRP_{p != n} B_p]                       (Alg. 1; Eq. 12)
  T_n = HADAMARD_{p != n} A_p^T A_p = ... B_p^T B_p     (Eq. 9)
  B_n <- H_n T_n^{-1}                                  (Eq. 14 in core space)
and finally A_n = U_n B_n (Eq. 13).  The textbook form on an explicit tensor
(Eq. 6) is the same function applied to Y~ itself, which the tests use to pin
the core-space form.
"""
from __future__ import annotations

import math

import numpy as np

from .tucker import khatri_rao, unfold


def mttkrp(G: np.ndarray, Bs, n: int) -> np.ndarray:
    """H_n = G_(n) [KRP_{p != n} B_p] with the Khatri-Rao product formed
    (Alg. 1, the matricised-tensor product; Eq. 12).  Pinned by brute force in tests."""
    N = G.ndim
    return unfold(G, n) @ khatri_rao([Bs[p] for p in range(N) if p != n])


def hadamard_grams(Bs, n: int) -> np.ndarray:
    """T_n = HADAMARD_{p != n} B_p^T B_p (Eq. 9).  Pinned: equals the Gram of
    the explicit Khatri-Rao product of the other factors."""
    R = Bs[0].shape[1]
    T = np.ones((R, R))
    for p, B in enumerate(Bs):
        if p != n:
            T = T * (B.T @ B)
    return T


def solve_normal(H: np.ndarray, T: np.ndarray):
    """X = H T^{-1} for symmetric positive semidefinite T (Eq. 6 / Eq. 14).

    Cholesky when every pivot exceeds R * eps * max_j T_jj; otherwise the
    pseudo-inverse from the eigendecomposition of T with cutoff
    R * eps * lambda_max (the paper writes the inverse; both thresholds are
    this implementation's reading for a singular Hadamard product of Grams).
    Returns (X, used_pinv).  Pinned: X T = H on an SPD T; LAPACK's pinv on a
    singular one.
    """
    R = T.shape[0]
    L = np.zeros_like(T)
    ok = True
    tiny = R * np.finfo(np.float64).eps * max(float(np.max(np.diag(T))), 0.0)
    for j in range(R):
        d = T[j, j] - np.dot(L[j, :j], L[j, :j])
        if not d > tiny:
            ok = False
            break
        L[j, j] = math.sqrt(d)
        for i in range(j + 1, R):
            L[i, j] = (T[i, j] - np.dot(L[i, :j], L[j, :j])) / L[j, j]
    if ok:
        # X T = H  <=>  T X^T = H^T,  T = L L^T
        Yt = np.linalg.solve(L, H.T)
        return np.linalg.solve(L.T, Yt).T, False
    w, V = np.linalg.eigh(T)
    cut = R * np.finfo(np.float64).eps * max(w.max(), 0.0)
    winv = np.where(w > cut, 1.0 / np.where(w > cut, w, 1.0), 0.0)
    return H @ (V * winv[None, :]) @ V.T, True


def cp_full(lam, Bs) -> np.ndarray:
    """Dense [[lambda; B_1, ..., B_N]] (Eq. 2).  Pinned: brute-force sums."""
    Bs = [np.asarray(b, dtype=np.float64) for b in Bs]
    shape = tuple(b.shape[0] for b in Bs)
    R = Bs[0].shape[1]
    out = np.zeros(shape)
    for r in range(R):
        t = lam[r] * Bs[0][:, r]
        for b in Bs[1:]:
            t = np.multiply.outer(t, b[:, r])
        out += t
    return out


def _normalise(B: np.ndarray):
    lam = np.sqrt(np.sum(B * B, axis=0))
    safe = np.where(lam > 0, lam, 1.0)
    return B / safe[None, :], lam


def core_fit(normG2: float, inner: float, model2: float) -> float:
    """Fit = 1 - ||X - X^||_F / ||X||_F (Sec. III-B) from the identity
    ||X - X^||^2 = ||X||^2 - 2 <X, X^> + ||X^||^2.  Pinned: against the
    explicit residual of a converged run."""
    res2 = max(0.0, normG2 - 2.0 * inner + model2)
    return 1.0 - math.sqrt(res2) / math.sqrt(normG2)


def cp_als(G: np.ndarray, B_init, max_sweeps: int = 1000, tol: float = 1e-9):
    """Textbook CP-ALS (Eqs. 3-6, 9), applied to the Tucker core G.

    Sweeps modes 1..N in order (Gauss-Seidel); after each mode update the
    columns of B_n are scaled to unit 2-norm and the norms kept as lambda.
    After each sweep the fit is evaluated from the last mode's H and the
    Grams; the loop stops when |f_t - f_{t-1}| < tol * |f_{t-1}| or after
    max_sweeps.  Returns dict(B=normalised factors, lam, fit, sweeps, history).
    Pinned: textbook ALS on the explicit Y~ (Eq. 17), exact recovery of
    noise-free CP tensors, the fit of Table II and the noise floor.
    """
    G = np.asarray(G, dtype=np.float64)
    N = G.ndim
    Bs = [np.array(b, dtype=np.float64) for b in B_init]
    R = Bs[0].shape[1]
    lam = np.ones(R)
    nG2 = float(np.sum(G * G))
    hist = []
    fit_old = None
    sweeps = 0
    npinv = 0
    for sweep in range(1, max_sweeps + 1):
        sweeps = sweep
        for n in range(N):
            H = mttkrp(G, Bs, n)
            T = hadamard_grams(Bs, n)
            Bn, used = solve_normal(H, T)
            npinv += int(used)
            Bs[n], lam = _normalise(Bn)
        inner = float(np.sum(H * (Bs[N - 1] * lam[None, :])))
        gram = np.ones((R, R))
        for b in Bs:
            gram = gram * (b.T @ b)
        model2 = float(lam @ gram @ lam)
        fit = core_fit(nG2, inner, model2)
        hist.append(fit)
        if fit_old is not None and abs(fit - fit_old) < tol * abs(fit_old):
            break
        fit_old = fit
    return {"B": Bs, "lam": lam, "fit": hist[-1], "sweeps": sweeps, "history": hist,
            "inner": inner, "model2": model2, "normG2": nG2, "pinv_used": npinv}


def hals_rows(A0: np.ndarray, M: np.ndarray, T: np.ndarray) -> np.ndarray:
    """HALS update of A (Eq. 8): column by column, r = 1..R,
        a_r <- P_+( a_r + (m_r - A t_r) / t_rr ),
    with the columns already updated in this pass used for A (the projection
    applied to the updated column: the exact minimiser of the objective over
    column r with the others fixed).  Pinned: brute-force minimisation of the
    objective over each column on a grid; exact recovery of a noise-free
    nonnegative CP model."""
    A = np.array(A0, dtype=np.float64)
    for r in range(A.shape[1]):
        A[:, r] = np.maximum(0.0, A[:, r] + (M[:, r] - A @ T[:, r]) / T[r, r])
    return A


def mu_rows(A0: np.ndarray, M: np.ndarray, T: np.ndarray) -> np.ndarray:
    """Multiplicative update in the low-rank form (Eq. 15):
        A <- A (*) P_+(M) (/) (A T),
    elementwise; an entry whose denominator is not positive becomes 0.
    Pinned: an exact nonnegative factor is a fixed point; on nonnegative data
    the objective never rises (Lee and Seung); exact recovery."""
    A0 = np.asarray(A0, dtype=np.float64)
    D = A0 @ T
    out = np.zeros_like(A0)
    pos = D > 0.0
    out[pos] = A0[pos] * np.maximum(M, 0.0)[pos] / D[pos]
    return out


def soft_threshold(X: np.ndarray, c: float) -> np.ndarray:
    """S_c(x) = sign(x) max(|x| - c, 0), elementwise (Eq. 16): the minimiser
    of (z - x)^2 / 2 + c |z| (pinned by brute force)."""
    X = np.asarray(X, dtype=np.float64)
    return np.sign(X) * np.maximum(np.abs(X) - c, 0.0)


def cp_als_nonneg(G: np.ndarray, Us, A_init, max_sweeps: int = 1000, tol: float = 1e-7, rule: str = "ls",
                  l1: float = 0.0, clip: bool = True):
    """FFCP with projected nonnegative LS updates on the Tucker format.

    For every mode (Alg. 1 with the LS rule of Eq. 14 followed by P_+ of Eq. 8):
      H_n = G_(n) [KRP_{p != n} B_p]        with B_p = U_p^T A_p   (Eqs. 12, 13)
      M_n = U_n H_n                          (~ Y_(n) B, Eq. 12)
      T_n = HADAMARD_{p != n} A_p^T A_p       (Eq. 9, the actual A_p)
      A_n <- max(0, M_n T_n^{-1}),  B_n <- U_n^T A_n
    Columns of A_n are scaled to unit norm (lambda); an all-zero column is
    replaced by the constant unit vector with lambda_r = 0.  The fit is taken
    against Y~ = [[G; U]]:  <Y~, [[A]]> = <G, [[B]]>, ||[[A]]||^2 from A's Grams.

    rule "hals" (Eq. 8) and "mu" (Eq. 15) replace the projected solve by one
    pass of `hals_rows` / `mu_rows` from the current iterate of the mode,
    A_n diag(lambda) (the model [[lambda; A]] with lambda on the factor being
    updated), with the same M_n and T_n.

    l1 > 0 (rule "ls"): the l1-regularised update of Eq. 16, A_n <- S_c(A_n)
    applied to the LS solution before the projection; clip=False drops the
    projection P_+ (the sparse but signed form).

    Pinned: exact recovery of noise-free nonnegative CP models (every rule);
    with HALS and MU, the fit of Table III's 200^3 case, both against the
    paper's band and against the first-order noise floor of a least-squares
    fit at 10 dB.
    """
    G = np.asarray(G, dtype=np.float64)
    N = G.ndim
    As = [np.array(a, dtype=np.float64) for a in A_init]
    Us = [np.asarray(u, dtype=np.float64) for u in Us]
    Bs = [Us[n].T @ As[n] for n in range(N)]
    R = As[0].shape[1]
    lam = np.ones(R)
    nG2 = float(np.sum(G * G))
    hist = []
    fit_old = None
    sweeps = 0
    for sweep in range(1, max_sweeps + 1):
        sweeps = sweep
        for n in range(N):
            H = mttkrp(G, Bs, n)
            M = Us[n] @ H
            T = hadamard_grams(As, n)
            if rule == "ls":
                An, _ = solve_normal(M, T)
                if l1 > 0.0:
                    An = soft_threshold(An, l1)
                if clip:
                    An = np.maximum(An, 0.0)
            elif rule == "hals":
                An = hals_rows(As[n] * lam[None, :], M, T)
            elif rule == "mu":
                An = mu_rows(As[n] * lam[None, :], M, T)
            else:
                raise ValueError(rule)
            An, lam = _normalise(An)
            zero = lam == 0
            if np.any(zero):
                An[:, zero] = 1.0 / math.sqrt(An.shape[0])
            As[n] = An
            Bs[n] = Us[n].T @ An
        inner = float(np.sum(H * (Bs[N - 1] * lam[None, :])))
        gram = np.ones((R, R))
        for a in As:
            gram = gram * (a.T @ a)
        model2 = float(lam @ gram @ lam)
        fit = core_fit(nG2, inner, model2)
        hist.append(fit)
        if fit_old is not None and abs(fit - fit_old) < tol * abs(fit_old):
            break
        fit_old = fit
    return {"A": As, "B": Bs, "lam": lam, "fit": hist[-1], "sweeps": sweeps, "history": hist,
            "inner": inner, "model2": model2, "normG2": nG2}


def lift(Us, Bs, lam):
    """A_n = U_n B_n (Eq. 13 / Eq. 17), lambda absorbed into A_N (Sec. II).
    Pinned: exact recovery of noise-free CP tensors by explicit residual."""
    A = [np.asarray(u, dtype=np.float64) @ np.asarray(b, dtype=np.float64) for u, b in zip(Us, Bs)]
    A[-1] = A[-1] * np.asarray(lam)[None, :]
    return A


def hosvd_init(G: np.ndarray, R: int):
    """Leading R left singular vectors of G_(n) for every n (HOSVD of the core,
    Sec. II), each column's sign fixed so its largest-magnitude entry is
    positive.  Needs R <= R_n.  Pinned: spans the leading eigenvectors of
    G_(n) G_(n)^T."""
    out = []
    for n in range(G.ndim):
        Un, _, _ = np.linalg.svd(unfold(G, n), full_matrices=False)
        V = Un[:, :R].copy()
        idx = np.argmax(np.abs(V), axis=0)
        s = np.sign(V[idx, np.arange(R)])
        s[s == 0] = 1.0
        out.append(V * s[None, :])
    return out


def congruence(A_true, A_est) -> float:
    """Factor congruence after permutation / scale alignment: columns are
    matched by the Hungarian method on prod_n |cos(a_nr, a^_ns)| and the
    minimum over matched pairs is returned.  Pinned: 1 under column
    permutation and scaling; cos(theta) for one column turned by theta."""
    from scipy.optimize import linear_sum_assignment

    R = A_true[0].shape[1]
    C = np.ones((R, R))
    for a, b in zip(A_true, A_est):
        an = a / np.linalg.norm(a, axis=0, keepdims=True)
        bn = b / np.maximum(np.linalg.norm(b, axis=0, keepdims=True), 1e-300)
        C = C * np.abs(an.T @ bn)
    ri, ci = linear_sum_assignment(-C)
    return float(C[ri, ci].min())


def sir_db(A_true, A_est):
    """Signal-to-interference ratio of every recovered component, in dB
    (Sec. V-A, footnote to the 10^4-dimension experiment): both columns are
    brought to zero mean and unit variance, then
        SIR(a, a^) = -20 log10(||a - a^|| / ||a||),
    the footnote's ratio with the sign that makes a better estimate score
    higher.  Columns are matched as in `congruence`, and the sign of each
    estimate is aligned with its match.  Returns the list over all modes and
    components.  Pinned: a planted perturbation of known size gives the
    closed-form value."""
    from scipy.optimize import linear_sum_assignment

    def zs(x):
        x = np.asarray(x, dtype=np.float64)
        x = x - x.mean(axis=0, keepdims=True)
        return x / np.maximum(x.std(axis=0, keepdims=True), 1e-300)

    Z = [zs(a) for a in A_true]
    Zh = [zs(b) for b in A_est]
    R = Z[0].shape[1]
    C = np.ones((R, R))
    for a, b in zip(Z, Zh):
        C = C * np.abs(a.T @ b) / a.shape[0]
    ri, ci = linear_sum_assignment(-C)
    out = []
    for a, b in zip(Z, Zh):
        for r, c in zip(ri, ci):
            e = b[:, c] if a[:, r] @ b[:, c] >= 0.0 else -b[:, c]
            out.append(-20.0 * math.log10(max(np.linalg.norm(a[:, r] - e), 1e-300) / np.linalg.norm(a[:, r])))
    return out

