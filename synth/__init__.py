"""Seeded synthetic inputs shared by the CUDA path, the oracle, the tests and the bench.

This module draws inputs only; it holds none of the decomposition arithmetic
(no sketch, no orthonormalisation, no TTM, no ALS).  What it produces:

* CP-model data tensors with Gaussian noise at a given SNR, the data model of
  the paper's synthetic experiments (Sec. V-A, CP model of Eq. 2 plus i.i.d.
  Gaussian noise; nonnegative variant with clipped values), and the sparse
  nonnegative factors of its nonnegative CPD experiments (exponential
  entries, a fixed share of them set to zero).
* Exact multilinear-rank tensors (Tucker model, Eq. 1) for exact-recovery tests.
* The small Gaussian matrices W_k^(n) whose Khatri-Rao product is the random
  test matrix Omega_n of the range finder (Sec. IV-A, step 1).  They are drawn
  N(0,1) and stored rounded to the nearest BF16 value, so every precision form
  of the sketch (FP64, FP32, BF16 tensor cores) consumes the identical Omega.
* Initial CP factors for ALS (the first step of Alg. 1).

Every draw is keyed by (seed, tag...) through numpy's SeedSequence, so a draw
does not depend on which other draws were made before it.  Big tensors are
generated slab by slab on the GPU with torch (input generation only); a slab
can be copied back to the host to feed the oracle.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# tags that separate independent random streams drawn from one seed
TAG_FACTORS = 1
TAG_NOISE = 2
TAG_SKETCH = 3
TAG_INIT = 4
TAG_TUCKER = 5
TAG_MASK = 6
TAG_SKETCH_SHARED = 8
TAG_REFINE = 9
TAG_SPARSE_NN = 10
TAG_DENSE_OMEGA = 11

OMEGA_SEED_XOR = 0x9E3779B97F4A7C15


def rng(seed: int, *tags: int) -> np.random.Generator:
    words = [int(seed) & 0xFFFFFFFF, (int(seed) >> 32) & 0xFFFFFFFF] + [int(t) for t in tags]
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence(words)))


def round_bf16(x) -> np.ndarray:
    """Round to the nearest BF16 value (ties to even), returned as float64.

    BF16 keeps an 8-bit significand; frexp gives x = m * 2**e with m in
    [0.5, 1), so m * 2**8 rounded to an integer is the significand.
    """
    x = np.asarray(x, dtype=np.float64)
    m, e = np.frexp(x)
    return np.ldexp(np.rint(m * 256.0) / 256.0, e)


def correlated_factor(r: np.random.Generator, I: int, R: int, rho: float,
                      dist: str = "normal") -> np.ndarray:
    """I x R factor whose columns have pairwise correlation rho.

    A = X L^T with L L^T = (1 - rho) I + rho 11^T and X i.i.d.; for rho = 0 the
    columns are just i.i.d. draws.
    """
    if dist == "normal":
        X = r.standard_normal((I, R))
    elif dist == "uniform":
        X = r.random((I, R))
    else:
        raise ValueError(dist)
    if rho == 0.0:
        return X
    C = (1.0 - rho) * np.eye(R) + rho * np.ones((R, R))
    L = np.linalg.cholesky(C)
    return X @ L.T


def cp_factors(shape, R: int, seed: int, dist: str = "normal", rho: float = 0.0):
    r = rng(seed, TAG_FACTORS)
    return [correlated_factor(r, I, R, rho, dist) for I in shape]


def sparse_exponential_factors(shape, R: int, seed: int, mean: float = 10.0, zero_frac: float = 0.1):
    """Nonnegative CP factors of the data model in Sec. V-A ("Simulations on
    Nonnegative CPD"): entries i.i.d. exponential with the given mean, then
    round(zero_frac * I * R) entries of each factor, chosen uniformly without
    replacement, set to zero."""
    out = []
    for n, I in enumerate(shape):
        r = rng(seed, TAG_SPARSE_NN, n)
        A = r.exponential(mean, (I, R))
        k = int(round(zero_frac * I * R))
        A.reshape(-1)[r.choice(I * R, k, replace=False)] = 0.0
        out.append(A)
    return out


def cp_dense(factors) -> np.ndarray:
    """Dense CP tensor sum_r a1_r o a2_r o ... (row-major, last mode fastest)."""
    N = len(factors)
    R = factors[0].shape[1]
    shape = tuple(f.shape[0] for f in factors)
    out = np.zeros(shape)
    for r in range(R):
        t = factors[0][:, r]
        for n in range(1, N):
            t = np.multiply.outer(t, factors[n][:, r])
        out += t
    return out


def noise_sigma(signal_energy: float, numel: int, snr_db: float) -> float:
    """Noise std so that ||Y*||^2 / E||E||^2 = 10^(SNR/10)."""
    return math.sqrt(signal_energy * 10.0 ** (-snr_db / 10.0) / numel)


def add_noise(Ystar: np.ndarray, snr_db: float | None, seed: int, clip0: bool = False) -> np.ndarray:
    if snr_db is None:
        Y = Ystar.copy()
    else:
        s = noise_sigma(float(np.sum(Ystar * Ystar)), Ystar.size, snr_db)
        Y = Ystar + s * rng(seed, TAG_NOISE).standard_normal(Ystar.shape)
    if clip0:
        np.maximum(Y, 0.0, out=Y)
    return Y


def tucker_dense(shape, ranks, seed: int) -> np.ndarray:
    """Tensor of exact multilinear rank `ranks` (Tucker model, Eq. 1)."""
    r = rng(seed, TAG_TUCKER)
    core = r.standard_normal(tuple(ranks))
    out = core
    for n, (I, Rn) in enumerate(zip(shape, ranks)):
        U = r.standard_normal((I, Rn))
        out = np.moveaxis(np.tensordot(U, out, axes=([1], [n])), 0, n)
    return out


def omega_seed(w: "Workload") -> int:
    """Seed of a workload's test matrices when the library draws them
    (tdk_tucker_desc.seed): the workload seed with the sketch offset."""
    return (int(w.seed) ^ OMEGA_SEED_XOR) & ((1 << 64) - 1)


def sketch_matrices(shape, Rt, seed: int, shared: bool = False):
    """W[n][k] (k != n): I_k x Rt[n] i.i.d. N(0,1), rounded to BF16 values.

    Omega_n is the Khatri-Rao product of W[n][k] over k != n (never formed by
    the CUDA path).  W[n][n] is None.

    shared=True draws one matrix W_k (I_k x max Rt) per mode and uses it for
    every sketch: W[n][k] = W_k (its first Rt[n] columns where Rt[n] is
    narrower).  Every Omega_n is still a Khatri-Rao product of independent
    N(0,1) matrices, so each sketch has the distribution of the independent
    family; only the sketches of different modes become dependent.  Entries
    of equal width are the same array object (`device_sketch` uploads such an
    object once).
    """
    N = len(shape)
    if np.isscalar(Rt):
        Rt = [int(Rt)] * N
    base = int(seed) ^ OMEGA_SEED_XOR
    if shared:
        wmax = max(int(r) for r in Rt)
        Wk = [round_bf16(rng(base, TAG_SKETCH_SHARED, k).standard_normal((shape[k], wmax))) for k in range(N)]
        return [[None if k == n else (Wk[k] if int(Rt[n]) == wmax else np.ascontiguousarray(Wk[k][:, :Rt[n]]))
                 for k in range(N)] for n in range(N)]
    W = []
    for n in range(N):
        row = []
        for k in range(N):
            if k == n:
                row.append(None)
            else:
                row.append(round_bf16(rng(base, TAG_SKETCH, n, k).standard_normal((shape[k], Rt[n]))))
        W.append(row)
    return W


def dense_test_matrices(shape, Rt, seed: int, sequential: bool = False):
    """Dense Gaussian test matrices Omega_n, i.i.d. N(0,1), for the range
    finder as printed (Sec. IV-A, step 1): prod_{k != n} I_k rows for the
    all-mode sketch, or prod_{k<n} Rt_k prod_{k>n} I_k rows for Alg. 2's
    sequential form (modes before n already shrunk); Rt_n columns."""
    N = len(shape)
    out = []
    for n in range(N):
        rows = 1
        for k in range(N):
            if k != n:
                rows *= Rt[k] if (sequential and k < n) else shape[k]
        out.append(rng(seed, TAG_DENSE_OMEGA, n, int(sequential)).standard_normal((rows, Rt[n])))
    return out


def refine_matrices(Rt, seed: int, it: int):
    """Sketch matrices of refinement pass `it` (RandTucker2i): W[n][k]
    (k != n) is Rt[k] x Rt[n] i.i.d. N(0,1) rounded to BF16 values."""
    N = len(Rt)
    base = int(seed) ^ OMEGA_SEED_XOR
    return [[None if k == n else round_bf16(rng(base, TAG_REFINE, it, n, k).standard_normal((Rt[k], Rt[n])))
             for k in range(N)] for n in range(N)]


def random_factors(shape, Rt, seed: int):
    """RandTucker2i's starting factors: I_n x Rt_n i.i.d. N(0,1)."""
    return [rng(seed, TAG_REFINE, 99, n).standard_normal((shape[n], Rt[n])) for n in range(len(shape))]


def device_sketch(W, device):
    """W[n][k] as torch tensors on `device`; an array object that occurs more
    than once (a shared family) becomes one tensor."""
    import torch

    seen = {}
    out = []
    for row in W:
        r = []
        for x in row:
            if x is None:
                r.append(None)
                continue
            if id(x) not in seen:
                seen[id(x)] = torch.as_tensor(x, device=device)
            r.append(seen[id(x)])
        out.append(r)
    return out


def init_factors(dims, R: int, seed: int, dist: str = "normal"):
    """Initial CP factors (one per entry of dims), i.i.d. N(0,1) or U[0,1]."""
    out = []
    for n, I in enumerate(dims):
        r = rng(seed, TAG_INIT, n)
        out.append(r.standard_normal((I, R)) if dist == "normal" else r.random((I, R)))
    return out


TAG_MLP = 7


def mlp_init_params(N: int, Rt: int, hidden: int, seed: int, hosvd_start: bool = False,
                    out_scale: float = 1.0) -> np.ndarray:
    """Initial parameter vector of the learned initialiser's MLP (layout
    W1, b1, W2, b2, W3, b3 as in the C header): weights i.i.d.
    N(0, 1 / fan_in), biases zero, as float32.  With hosvd_start the output
    bias holds an identity block per mode (in canonical coordinates the
    leading singular vectors of the core: the HOSVD start of ALS) and the
    output weights are scaled by out_scale, so training starts from the HOSVD
    initialisation and learns corrections to it."""
    din, dout = Rt ** N, N * Rt * Rt
    r = rng(seed, TAG_MLP)
    parts = []
    for li, (fan_in, fan_out) in enumerate(((din, hidden), (hidden, hidden), (hidden, dout))):
        W = r.standard_normal((fan_out, fan_in)) / math.sqrt(fan_in)
        b = np.zeros(fan_out)
        if li == 2 and hosvd_start:
            W = W * out_scale
            b = np.concatenate([np.eye(Rt).ravel() for _ in range(N)]) * 0.5
        parts.append(W.ravel())
        parts.append(b)
    return np.concatenate(parts).astype(np.float32)


TAG_LEARNED = 99


def learned_init_workload(k: int, split: int, shape=None, Rt: int | None = None, rmin: int = 8) -> "Workload":
    """Sample k of the learned-initialiser workload (split 1: training, 2:
    held out): 3-way CP data with rank R ~ U{rmin..Rt}, column correlation
    ~ U[0, 0.9], SNR ~ U[10, 40] dB; Tucker ranks Rt with p = 0; ALS rank R."""
    import dataclasses

    base = WORKLOADS["c5"]
    shape = tuple(base.shape if shape is None else shape)
    Rt = base.Rt[0] if Rt is None else int(Rt)
    seed = base.seed + split * 1000000 + k
    r = rng(seed, TAG_LEARNED)
    R = int(r.integers(rmin, Rt + 1))
    return dataclasses.replace(base, name=f"{base.name}_{split}_{k}", shape=shape, R_cp=R,
                               rho=float(r.uniform(0, 0.9)), snr_db=float(r.uniform(10, 40)), seed=seed,
                               ranks=(Rt,) * len(shape), p=0, als_R=R)


# --------------------------------------------------------------------------
# The five workloads (sizes, ranks and data model of the synthetic runs).
# --------------------------------------------------------------------------
@dataclass
class Workload:
    name: str
    shape: tuple
    R_cp: int               # CP rank of the planted data
    ranks: tuple            # Tucker ranks R_n
    p: int                  # oversampling
    dtype: str              # storage type of Y: f64 / f32 / bf16
    snr_db: float | None
    seed: int
    dist: str = "normal"
    rho: float = 0.0
    clip0: bool = False
    nonneg: bool = False
    als_R: int = 0
    als_max_sweeps: int = 1000
    als_tol: float = 1e-7
    extra: dict = field(default_factory=dict)

    @property
    def N(self):
        return len(self.shape)

    @property
    def Rt(self):
        return tuple(r + self.p for r in self.ranks)

    @property
    def numel(self):
        return int(np.prod(self.shape))

    @property
    def itemsize(self):
        return {"f64": 8, "f32": 4, "bf16": 2}[self.dtype]


WORKLOADS = {
    "c1": Workload("cp3_100_f64", (100, 100, 100), 5, (5, 5, 5), 5, "f64", 30.0, 0,
                   als_R=5, als_max_sweeps=100, als_tol=1e-9),
    "c2": Workload("cp3_1000_f32", (1000, 1000, 1000), 10, (10, 10, 10), 10, "f32", 20.0, 2,
                   rho=0.5, als_R=10, als_max_sweeps=1000, als_tol=1e-7),
    "c3": Workload("cp4_200_f32_nonneg", (200, 200, 200, 200), 20, (20, 20, 20, 20), 10, "f32", 25.0, 3,
                   dist="uniform", clip0=True, nonneg=True, als_R=20, als_max_sweeps=1000, als_tol=1e-7),
    "c4": Workload("cp3_3000_bf16", (3000, 3000, 3000), 40, (40, 40, 40), 20, "bf16", 15.0, 4,
                   als_R=40, als_max_sweeps=1000, als_tol=1e-7),
    "c5": Workload("cp3_300_f32_learned_init", (300, 300, 300), 20, (20, 20, 20), 0, "f32", None, 10,
                   als_R=20, als_max_sweeps=1000, als_tol=1e-7),
}


def scaled(w: Workload, shape) -> Workload:
    """Same data model at another shape (for CPU-sized parity cases)."""
    d = dict(w.__dict__)
    d["shape"] = tuple(shape)
    d["name"] = w.name + "_at_" + "x".join(str(s) for s in shape)
    d["extra"] = dict(w.extra)
    return Workload(**d)


def host_tensor(w: Workload) -> np.ndarray:
    """The workload's data tensor on the host, float64 values already rounded
    to the storage type (for sizes that fit comfortably in host memory)."""
    A = cp_factors(w.shape, w.R_cp, w.seed, w.dist, w.rho)
    Y = add_noise(cp_dense(A), w.snr_db, w.seed, w.clip0)
    return to_storage(Y, w.dtype)


def to_storage(Y: np.ndarray, dtype: str) -> np.ndarray:
    if dtype == "f64":
        return np.asarray(Y, dtype=np.float64)
    if dtype == "f32":
        return np.asarray(Y, dtype=np.float32).astype(np.float64)
    if dtype == "bf16":
        return round_bf16(np.asarray(Y, dtype=np.float32).astype(np.float64))
    raise ValueError(dtype)


def device_tensor(w: Workload, device="cuda", slab: int = 0):
    """Generate the workload's tensor directly in GPU memory, slab by slab
    along mode 1 (input generation only; never timed).

    Y* = sum_r a1_r o ... o aN_r with host-drawn factors; the noise comes from
    torch's generator reseeded per slab, so any slab can be regenerated alone.
    Its std is set from ||Y*||^2 = 1^T (hadamard_n A_n^T A_n) 1.
    Returns (Y, factors).
    """
    import torch

    tdt = {"f64": torch.float64, "f32": torch.float32, "bf16": torch.bfloat16}[w.dtype]
    A = cp_factors(w.shape, w.R_cp, w.seed, w.dist, w.rho)
    gram = np.ones((w.R_cp, w.R_cp))
    for a in A:
        gram *= a.T @ a
    energy = float(gram.sum())
    sigma = 0.0 if w.snr_db is None else noise_sigma(energy, w.numel, w.snr_db)
    cdt = torch.float64 if w.dtype == "f64" else torch.float32
    At = [torch.as_tensor(a, dtype=cdt, device=device) for a in A]
    rest = int(np.prod(w.shape[1:]))
    Y = torch.empty(w.shape, dtype=tdt, device=device)
    # Khatri-Rao of modes 2..N as a (rest x R) operand; for big modes do it per sub-slab
    if slab <= 0:
        slab = max(1, min(w.shape[0], (1 << 26) // max(rest, 1)))
    g = torch.Generator(device=device)
    tail = At[1:]
    for i0 in range(0, w.shape[0], slab):
        i1 = min(w.shape[0], i0 + slab)
        # Y*[i, rest] = sum_r A1[i,r] * prod_{n>=2} An[i_n, r]
        K = tail[0]
        for t in tail[1:]:
            K = (K[:, None, :] * t[None, :, :]).reshape(-1, w.R_cp)
        blk = At[0][i0:i1] @ K.T
        if sigma > 0:
            g.manual_seed((int(w.seed) * 1000003 + i0) & 0x7FFFFFFFFFFFFFFF)
            blk += sigma * torch.randn(blk.shape, generator=g, device=device, dtype=cdt)
        if w.clip0:
            blk.clamp_(min=0)
        Y[i0:i1] = blk.reshape((i1 - i0,) + tuple(w.shape[1:])).to(tdt)
    return Y, A
