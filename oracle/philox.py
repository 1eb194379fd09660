"""Oracle: the seeded test matrices W_k^(n) of the all-mode sketch.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Sec. IV-A draws Gaussian test matrices and Sec. IV-B has the workers share
the seed of the generator instead of the matrices.  The library draws every
entry (i, r) of W_k^(n) from (seed, n, k, i, r) alone, with the counter-based
generator Philox4x32-10 of Salmon, Moraes, Dror and Shaw (SC'11); this module
is an independent implementation of the same definition:
  key = (seed mod 2^32, seed div 2^32), counter = (r, i mod 2^32, i div 2^32,
  256 n + k); ten rounds, each multiplying words 0 and 2 by 0xD2511F53 and
  0xCD9E8D57 (high and low halves of the 64-bit products), swapping and mixing
  in the key, the key bumped by 0x9E3779B9 and 0xBB67AE85 between rounds;
  a = (x0 2^32 + x1) div 2^11, b = (x2 2^32 + x3) div 2^11,
  u1 = (a + 1/2) 2^-53, u2 = b 2^-53, z = sqrt(-2 ln u1) cos(2 pi u2),
  and the entry is z rounded to the nearest BF16 value (ties to even).
Pins (tests/test_oracle_pins.py): the published known-answer vectors of
Philox4x32-10, the moments and the independence of the drawn values, the
BF16 rounding against its definition, and row blocks drawn alone.
"""
from __future__ import annotations

import numpy as np

_M0, _M1 = np.uint64(0xD2511F53), np.uint64(0xCD9E8D57)
_W0, _W1 = np.uint64(0x9E3779B9), np.uint64(0xBB67AE85)
_LO = np.uint64(0xFFFFFFFF)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Ten Philox4x32 rounds on arrays of counters (uint32 values held in
    uint64) under the key (k0, k1); returns the four output words."""
    c0, c1, c2, c3 = (np.asarray(x, dtype=np.uint64) & _LO for x in (c0, c1, c2, c3))
    k0 = np.asarray(k0, dtype=np.uint64) & _LO
    k1 = np.asarray(k1, dtype=np.uint64) & _LO
    for _ in range(10):
        p0 = _M0 * c0
        p1 = _M1 * c2
        c0, c1, c2, c3 = ((p1 >> np.uint64(32)) ^ c1 ^ k0, p1 & _LO, (p0 >> np.uint64(32)) ^ c3 ^ k1, p0 & _LO)
        k0 = (k0 + _W0) & _LO
        k1 = (k1 + _W1) & _LO
    return c0, c1, c2, c3


def round_bf16(x):
    """Nearest BF16 value (8 significant bits, ties to even), as float64."""
    x = np.asarray(x, dtype=np.float64)
    m, e = np.frexp(x)
    return np.ldexp(np.rint(m * 256.0) / 256.0, e)


def normals(seed: int, n: int, k: int, rows, cols: int, row0: int = 0):
    """Unrounded FP64 normals of entries (row0 + i, r), i < rows, r < cols."""
    i = np.arange(row0, row0 + rows, dtype=np.uint64)[:, None] * np.ones((1, cols), dtype=np.uint64)
    r = np.arange(cols, dtype=np.uint64)[None, :] * np.ones((rows, 1), dtype=np.uint64)
    seed = int(seed) & ((1 << 64) - 1)
    x0, x1, x2, x3 = philox4x32_10(r, i & _LO, i >> np.uint64(32), np.uint64(256 * n + k), seed & 0xFFFFFFFF,
                                   seed >> 32)
    a = ((x0 << np.uint64(32)) | x1) >> np.uint64(11)
    b = ((x2 << np.uint64(32)) | x3) >> np.uint64(11)
    u1 = (a.astype(np.float64) + 0.5) * 2.0 ** -53
    u2 = b.astype(np.float64) * 2.0 ** -53
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


def sketch_matrices(seed: int, dims, Rt, row0=None, rows=None):
    """W[n][k] = the seeded W_k^(n) [rows_k x Rt_n] (rows_k = dims[k] unless
    given; first row at global index row0[k]); W[n][n] is None."""
    N = len(dims)
    row0 = [0] * N if row0 is None else list(row0)
    rows = list(dims) if rows is None else list(rows)
    return [[None if k == n else round_bf16(normals(seed, n, k, rows[k], Rt[n], row0[k])) for k in range(N)]
            for n in range(N)]
