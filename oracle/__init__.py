"""CPU FP64 oracle for the randomized Tucker + FFCP path.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import or run
anything in this package.  It shares no code with the CUDA library: no
kernels, headers, helpers or constant tables, and neither imports the other.
Inputs come from the seeded generators in ``synth`` (or from the paper).

Everything is plain numpy in float64, written to follow the paper's
definitions and algorithm steps in their order; a library primitive (matmul,
einsum, a small linear solve or eigendecomposition) may serve as one step.

Conventions (readings where the paper's MATLAB convention is implicit):
  * tensors are row-major, last mode fastest;
  * the mode-n unfolding Y_(n) has row i_n and columns the remaining indices
    in row-major order (slowest first);
  * the Khatri-Rao product over k != n orders its factors slowest first,
    (A (.) B)[(i, j), r] = A[i, r] B[j, r] with j fastest, which matches the
    column order of Y_(n).

Parity status of each function is stated in its docstring.  "parity unpinned"
marks a function with no pin independent of itself.
"""
from .tucker import (unfold, fold, khatri_rao, sketch, sketch_row, householder_qr,
                     ttm, tucker_core, rand_tucker, tucker_full, norm2, hosvd_factors, refine_pass,
                     rand_tucker_2i, evd_orth, rand_tucker_dense, rand_tucker_seq, seq_test_matrices,
                     rand_tucker_seq_krp, grid_blocks,
                     sketch_share, core_share, rand_tucker_grid)
from .cpals import (mttkrp, hadamard_grams, cp_full, cp_als, cp_als_nonneg, core_fit,
                    lift, congruence, sir_db, solve_normal, hosvd_init, hals_rows, mu_rows, soft_threshold)
from . import mlp
from . import philox

__all__ = [
    "unfold", "fold", "khatri_rao", "sketch", "sketch_row", "householder_qr", "ttm",
    "tucker_core", "rand_tucker", "hosvd_factors", "refine_pass", "rand_tucker_2i", "evd_orth",
    "rand_tucker_dense", "rand_tucker_seq", "seq_test_matrices", "rand_tucker_seq_krp", "grid_blocks", "sketch_share", "core_share", "rand_tucker_grid", "tucker_full", "norm2", "mttkrp", "hadamard_grams",
    "cp_full", "cp_als", "cp_als_nonneg", "core_fit", "lift", "congruence", "sir_db", "solve_normal",
    "hosvd_init", "hals_rows", "mu_rows", "soft_threshold", "mlp", "philox",
]
