"""The sharded form of Sec. IV-B through the library on one GPU: two worker
processes, each holding a slab of mode 1 (61 rows: 31 + 30), exchange their
shares through gloo on the host (no kernel waits on another process).
Both workers end with the same core and factors, and these equal the
one-process library result on the same tensor and test matrices, within the
tolerance of the form, and the oracle's sub-tensor form."""
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

import oracle
import synth
from helpers import DT_CODE, dev_tensor, dev_W, host, small_problem

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, HERE)
from sharded_worker import P, R, RANKS, SEED, SHAPE  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("dtype,prec,seeded", [("f64", "simt", False), ("f32", "tc", True), ("bf16", "tc", False)])
def test_two_workers_match_one_process_and_oracle(tmp_path, dtype, prec, seeded):
    import torch

    import paper_1412_1885_gb300 as t
    from paper_1412_1885_gb300 import build

    build.build()
    out = str(tmp_path / "w")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr=127.0.0.1", f"--master-port={_free_port()}", os.path.join(HERE, "sharded_worker.py"), out,
           dtype, prec, "1" if seeded else "0"]
    env = dict(os.environ, OMP_NUM_THREADS="1")
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600, env=env)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    res = [np.load(f"{out}_{k}.npz") for k in range(2)]
    assert (int(res[0]["lo"]), int(res[0]["hi"]), int(res[1]["lo"]), int(res[1]["hi"])) == (0, 31, 31, 61)
    # both workers hold the same results, bit for bit
    for key in ("G", "U", "A", "normY2", "fit"):
        assert np.array_equal(res[0][key], res[1][key]), key
    # one process, same tensor and test matrices
    Y, W, _ = small_problem(SHAPE, RANKS, P, seed=31, dtype=dtype, R_cp=R)
    Rt = [x + P for x in RANKS]
    Wuse = oracle.philox.sketch_matrices(SEED, SHAPE, Rt) if seeded else W
    ctx = t.Context(0)
    B0 = [torch.as_tensor(b, device="cuda") for b in synth.init_factors(Rt, R, 5)]
    one = t.decompose(ctx, dev_tensor(Y, dtype), None if seeded else dev_W(W), RANKS, P, R, prec, max_sweeps=40,
                      tol=0.0, B0=B0, seed=SEED)
    G1 = host(one["G"])
    gb = oracle.tucker_core(np.abs(Y), [np.abs(host(u)) for u in one["U"]])
    tol = 1e-11 if dtype == "f64" else 5e-5
    assert np.all(np.abs(res[0]["G"] - G1) <= tol * gb + 1e-300)
    assert abs(float(res[0]["normY2"]) - float(one["normY2"].item())) <= 1e-6 * float(one["normY2"].item())
    # oracle: the sub-tensor form on the same slabs and test matrices
    ref = oracle.rand_tucker_grid(Y, Wuse, (2, 1, 1))
    e_sh = np.sqrt(max(0.0, float(res[0]["normY2"]) - float(np.sum(res[0]["G"] ** 2))) / float(res[0]["normY2"]))
    e_or = np.sqrt(max(0.0, oracle.norm2(Y) - float(np.sum(ref["G"] ** 2))) / oracle.norm2(Y))
    assert abs(e_sh - e_or) <= (1e-10 if dtype == "f64" else 1e-5), (e_sh, e_or)
    A1 = [host(a) for a in one["A"]]
    sizes = [SHAPE[n] * R for n in range(3)]
    As = np.split(res[0]["A"], np.cumsum(sizes)[:-1])
    As = [a.reshape(SHAPE[n], R) for n, a in enumerate(As)]
    assert oracle.congruence(A1, As) > (1 - 1e-9 if dtype == "f64" else 0.999)
    ctx.close()
    assert DT_CODE[dtype] in (0, 1, 2)
