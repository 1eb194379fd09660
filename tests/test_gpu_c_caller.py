"""A plain C program (tests/c/seeded_sketch.c) linked against libtdk.so calls
tucker_sketch with only the problem statement and a seed (W = NULL): the
library draws the test matrices itself.  Its sketches equal the oracle's on
the oracle's own draw of that seed, within the CUDA-core FP32 tolerance, and
its bases are the Householder bases of its sketches."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle
from helpers import TOL_SKETCH, basis_tol, sketch_abs_bound

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def _cuda_home():
    for c in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if c and os.path.exists(os.path.join(c, "include", "cuda_runtime.h")):
            return c
    pytest.skip("CUDA headers not found")


@pytest.fixture(scope="module")
def program(tmp_path_factory):
    from paper_1412_1885_gb300 import build

    build.build()
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    cuda = _cuda_home()
    libdir = os.path.join(ROOT, "paper_1412_1885_gb300")
    exe = str(tmp_path_factory.mktemp("c") / "seeded_sketch")
    lib64 = os.path.join(cuda, "lib64")
    if not os.path.isdir(lib64):
        lib64 = os.path.join(cuda, "lib")
    cmd = [cc, "-std=c99", "-O2", "-Wall", os.path.join(HERE, "c", "seeded_sketch.c"), "-I",
           os.path.join(ROOT, "include"), "-I", os.path.join(cuda, "include"), "-L", libdir, "-ltdk", "-L", lib64,
           "-lcudart", "-lm", f"-Wl,-rpath,{libdir}", f"-Wl,-rpath,{lib64}", "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return exe


@pytest.mark.parametrize("shape,ranks,p,seed", [((60, 50, 40), (5, 6, 7), 3, 42),
                                                ((33, 70, 65), (4, 4, 4), 4, 0xDEADBEEF12345678)])
def test_c_caller_with_a_seed_matches_oracle(program, tmp_path, shape, ranks, p, seed):
    out = str(tmp_path / "z.bin")
    args = [program, out, *map(str, shape), *map(str, ranks), str(p), str(seed)]
    r = subprocess.run(args, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    Rt = [x + p for x in ranks]
    raw = np.fromfile(out, dtype=np.float64)
    sizes = [shape[n] * Rt[n] for n in range(3)]
    assert raw.size == 2 * sum(sizes)
    parts, o = [], 0
    for rep in range(2):
        for n in range(3):
            parts.append(raw[o:o + sizes[n]].reshape(shape[n], Rt[n]))
            o += sizes[n]
    Z, U = parts[:3], parts[3:]
    a, b, c = np.meshgrid(*[np.arange(s, dtype=np.float64) for s in shape], indexing="ij")
    Y = (np.sin(0.37 * a + 0.11 * (b * c)) + 0.01 * (a - b + 2 * c) / shape[2]).astype(np.float32).astype(np.float64)
    W = oracle.philox.sketch_matrices(seed, shape, Rt)
    Zo, _ = oracle.sketch(Y, W)
    bnd = sketch_abs_bound(Y, W)
    tol = TOL_SKETCH[("f32", "simt")]
    for n in range(3):
        err = np.abs(Z[n] - Zo[n])
        assert np.all(err <= tol * bnd[n] + 1e-300), (n, float((err / bnd[n]).max()))
        assert np.abs(U[n] - oracle.householder_qr(Z[n])[0]).max() < basis_tol(Z[n])
