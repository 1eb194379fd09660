"""Learned FFCP initialiser: FP64 oracle of the canonicalisation, the MLP
forward and backward pass, the loss and the Adam update.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper has no learned part; its ALS starts from random or HOSVD factors
(the first step of Alg. 1).  The initialiser built here maps a compressed core G
(Alg. 2 output) to initial core-space factors B_n for FFCP.  Its definition:

canonicalise(G, colsums)
    For every mode n, V_n = the eigenvectors of G_(n) G_(n)^T (the left
    singular vectors of G_(n), HOSVD of the core), ordered by decreasing
    eigenvalue.  Column j of V_n gets the sign that makes colsum_n . v_j >= 0,
    where colsum_n = 1^T U_n are the column sums of the Tucker factor: the
    ambient vector U_n v_j then has a nonnegative entry sum, a rule that does
    not depend on the (random) basis U_n the sketch produced.
    S = G x_1 V_1^T ... x_N V_N^T / ||G||   (unit Frobenius norm).
input(S)
    x = sqrt(Rt^N) vec(S): the canonical core scaled to unit RMS.
forward(params, x)
    Z1 = x W1^T + b1,  H1 = gelu(Z1),  Z2 = H1 W2^T + b2,  H2 = gelu(Z2),
    O  = H2 W3^T + b3,  gelu(z) = z Phi(z) (exact, via erf).
    O holds N factors of Rt x Rt in canonical coordinates:
    O[(n Rt + i) Rt + r] = Bhat_n[i, r].
loss(O, S, R, T, alpha)
    Per sample, only the first R columns of every Bhat_n count:
    L = ||S - [[Bhat]]||^2 + alpha ||[[Bhat]] - [[T]]||^2, with T the target
    factors in the same coordinates (converged FFCP factors of the same core,
    see `canonical_target`); the batch loss is the mean over samples.  Both
    terms are invariant under a joint permutation of the R columns.
BF16 storage (the `bf16=True` form): the input x, the weights and the stored
    activations H1, H2 and the back-propagated dO, dZ2, dZ1 are BF16 values
    (rounded to nearest even) at exactly the points where the CUDA kernels
    store them; all arithmetic between those points is exact here (FP64).

Pins (tests/test_oracle_pins.py): central finite differences of `loss`
against `loss_grad` in the exact form (which covers `forward`, `gelu_grad`
and the parameter layout of `unpack`); the loss against a direct evaluation
of the Gram-identity formula; the invariance of `canonicalise` under a change
of Tucker basis (U_n -> U_n Q_n, G -> G x_n Q_n^T); for an exact CP core,
[[canonical_target]] equals the canonical core and `decanonicalise` undoes
the rotation; `network_input` has unit RMS; `gelu` against closed forms and
limits; Adam against its closed form for a constant gradient.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf

from .tucker import fold, unfold
from .cpals import cp_full

__all__ = ["mlp_dims", "param_sizes", "unpack", "canonicalise", "canonical_target", "network_input", "gelu",
           "gelu_grad", "linear", "activation", "delta", "dloss_dO",
           "forward", "loss", "loss_grad", "clip_grad", "adam_step", "decanonicalise"]


def _bf16(x):
    """Nearest BF16 value (ties to even) of every entry, as float64."""
    x = np.asarray(x, dtype=np.float64)
    m, e = np.frexp(x)
    return np.ldexp(np.rint(m * 256.0) / 256.0, e)


def mlp_dims(N: int, Rt: int, hidden: int):
    """(input, hidden, output) sizes: Rt^N core entries in, N Rt x Rt factors out."""
    return Rt ** N, hidden, N * Rt * Rt


def param_sizes(N: int, Rt: int, hidden: int):
    """Sizes of W1, b1, W2, b2, W3, b3 in the flat parameter vector, in order."""
    din, h, dout = mlp_dims(N, Rt, hidden)
    return [h * din, h, h * h, h, dout * h, dout]


def unpack(theta, N: int, Rt: int, hidden: int):
    """Split the flat parameter vector into W1 [h x in], b1, W2 [h x h], b2,
    W3 [out x h], b3 (row-major)."""
    din, h, dout = mlp_dims(N, Rt, hidden)
    shapes = [(h, din), (h,), (h, h), (h,), (dout, h), (dout,)]
    out, o = [], 0
    for s in shapes:
        n = int(np.prod(s))
        out.append(np.asarray(theta[o:o + n], dtype=np.float64).reshape(s))
        o += n
    return out


def canonicalise(G, colsums):
    """(S, V, normG): HOSVD rotation of the core with the sign rule above."""
    G = np.asarray(G, dtype=np.float64)
    N = G.ndim
    Vs = []
    for n in range(N):
        Gn = unfold(G, n)
        w, V = np.linalg.eigh(Gn @ Gn.T)
        V = V[:, np.argsort(-w, kind="stable")]
        s = np.asarray(colsums[n], dtype=np.float64) @ V
        V = V * np.where(s < 0.0, -1.0, 1.0)[None, :]
        Vs.append(V)
    S = G
    for n in range(N):
        shape = list(S.shape)
        shape[n] = Vs[n].shape[1]
        S = fold(Vs[n].T @ unfold(S, n), n, shape)
    nrm = math.sqrt(float(np.sum(G * G)))
    return S / nrm, Vs, nrm


def canonical_target(Bs, Vs, normG):
    """Target factors in canonical coordinates: T_n = V_n^T B_n, with the
    factors B_n of G = [[B_1, ..., B_N]] (weights absorbed) and the last one
    divided by ||G||, so that [[T]] approximates S."""
    T = [V.T @ np.asarray(B, dtype=np.float64) for V, B in zip(Vs, Bs)]
    T[-1] = T[-1] / normG
    return T


def network_input(S):
    """x = sqrt(Rt^N) vec(S) for a batch of canonical cores [batch, Rt, ..., Rt]."""
    S = np.asarray(S, dtype=np.float64)
    b = S.shape[0]
    X = S.reshape(b, -1)
    return X * math.sqrt(X.shape[1])


def decanonicalise(Bhat, Vs):
    """Core-space factors B_n = V_n Bhat_n (the column scale is irrelevant to ALS)."""
    return [V @ B for V, B in zip(Vs, Bhat)]


def gelu(z):
    """z * Phi(z), Phi the standard normal distribution function."""
    z = np.asarray(z, dtype=np.float64)
    return 0.5 * z * (1.0 + erf(z / math.sqrt(2.0)))


def gelu_grad(z):
    """d gelu / dz = Phi(z) + z phi(z)."""
    z = np.asarray(z, dtype=np.float64)
    return 0.5 * (1.0 + erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def _q(bf16: bool):
    return _bf16 if bf16 else (lambda a: np.asarray(a, dtype=np.float64))


def linear(H, W, b, bf16: bool = True):
    """One layer's pre-activation H W^T + b, the weights in storage precision."""
    return np.asarray(H, dtype=np.float64) @ _q(bf16)(W).T + b


def activation(Z, bf16: bool = True):
    """gelu(Z) in storage precision (the stored activation)."""
    return _q(bf16)(gelu(Z))


def delta(D_next, W, Z, bf16: bool = True):
    """Back-propagated pre-activation gradient (D_next W) * gelu'(Z) in
    storage precision, D_next the gradient of the next layer's output."""
    return _q(bf16)((np.asarray(D_next, dtype=np.float64) @ _q(bf16)(W)) * gelu_grad(Z))


def forward(theta, X, N: int, Rt: int, hidden: int, bf16: bool = True):
    """Batch forward pass; X [batch x Rt^N].  Returns (O, cache)."""
    W1, b1, W2, b2, W3, b3 = unpack(theta, N, Rt, hidden)
    X = _q(bf16)(X)
    Z1 = linear(X, W1, b1, bf16)
    H1 = activation(Z1, bf16)
    Z2 = linear(H1, W2, b2, bf16)
    H2 = activation(Z2, bf16)
    O = linear(H2, W3, b3, bf16)
    return O, {"X": X, "Z1": Z1, "H1": H1, "Z2": Z2, "H2": H2}


def _factors(o, N, Rt, R):
    return [o[n * Rt * Rt:(n + 1) * Rt * Rt].reshape(Rt, Rt)[:, :R] for n in range(N)]


def loss(O, S, R, T=None, alpha: float = 0.0):
    """Mean over the batch of ||S - [[Bhat]]||^2 + alpha ||[[Bhat]] - [[T]]||^2,
    each model tensor formed explicitly (Eq. 2 with unit weights)."""
    B = O.shape[0]
    N = S.ndim - 1
    Rt = S.shape[1]
    tot = 0.0
    for s in range(B):
        Bh = _factors(O[s], N, Rt, int(R[s]))
        M = cp_full(np.ones(int(R[s])), Bh)
        v = float(np.sum((S[s] - M) ** 2))
        if T is not None and alpha != 0.0:
            Mt = cp_full(np.ones(T[s][0].shape[1]), T[s])
            v += alpha * float(np.sum((M - Mt) ** 2))
        tot += v
    return tot / B


def dloss_dO(O, S, R, T, alpha):
    """Gradient of `loss` with respect to O (dense, exact)."""
    Bsz = O.shape[0]
    N = S.ndim - 1
    Rt = S.shape[1]
    dO = np.zeros_like(O)
    for s in range(Bsz):
        Rs = int(R[s])
        Bh = _factors(O[s], N, Rt, Rs)
        M = cp_full(np.ones(Rs), Bh)
        E = 2.0 * (M - S[s])
        if T is not None and alpha != 0.0:
            E = E + 2.0 * alpha * (M - cp_full(np.ones(T[s][0].shape[1]), T[s]))
        for n in range(N):
            # d<E, [[B]]>/dB_n = E_(n) KRP_{p != n} B_p (the Y_(n) B term of Eq. 5)
            others = [Bh[p] for p in range(N) if p != n]
            K = others[0]
            for P in others[1:]:
                K = np.einsum("ir,jr->ijr", K, P).reshape(-1, Rs)
            g = unfold(E, n) @ K
            blk = dO[s, n * Rt * Rt:(n + 1) * Rt * Rt].reshape(Rt, Rt)
            blk[:, :Rs] = g
    return dO / Bsz


def loss_grad(theta, X, S, R, N: int, Rt: int, hidden: int, T=None, alpha: float = 0.0, bf16: bool = True):
    """(loss, flat gradient, O) by back-propagation through `forward`.

    With bf16=True the back-propagated dO, dZ2 and dZ1 are rounded to BF16
    where the kernels store them; weight and bias gradients are exact sums of
    those rounded values against the (rounded) stored activations.
    """
    W1, b1, W2, b2, W3, b3 = unpack(theta, N, Rt, hidden)
    O, c = forward(theta, X, N, Rt, hidden, bf16)
    L = loss(O, S, R, T, alpha)
    dO = _q(bf16)(dloss_dO(O, S, R, T, alpha))
    gW3 = dO.T @ c["H2"]
    gb3 = dO.sum(axis=0)
    dZ2 = delta(dO, W3, c["Z2"], bf16)
    gW2 = dZ2.T @ c["H1"]
    gb2 = dZ2.sum(axis=0)
    dZ1 = delta(dZ2, W2, c["Z1"], bf16)
    gW1 = dZ1.T @ c["X"]
    gb1 = dZ1.sum(axis=0)
    g = np.concatenate([a.ravel() for a in (gW1, gb1, gW2, gb2, gW3, gb3)])
    return L, g, O


def clip_grad(g, clip: float):
    """Gradient-norm clipping (Pascanu, Mikolov and Bengio, ICML 2013): g
    scaled by min(1, clip / ||g||_2), the norm taken over all parameters;
    clip <= 0 leaves g as it is."""
    g = np.asarray(g, dtype=np.float64)
    if clip <= 0.0:
        return g
    n = float(np.sqrt(np.sum(g * g)))
    return g * (clip / n) if n > clip else g


def adam_step(theta, m, v, g, t: int, lr: float, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8):
    """One Adam update (Kingma and Ba, Algorithm 1), step t >= 1; returns
    (theta, m, v)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mh = m / (1.0 - beta1 ** t)
    vh = v / (1.0 - beta2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v
