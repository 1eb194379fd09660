"""Benchmark: one step = the whole path (all-mode sketch -> CholQR2 -> core ->
FFCP ALS to convergence -> lift) on one synthetic workload resident in HBM.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--config c4] [--prec tc]
    python bench.py --impl reference ...      (the FP64 oracle on the host cores)

value  = dense-tensor GB/s: algorithmic bytes 2 * itemsize * prod(I) (the two
         passes over Y: sketch, then core) per step / device time of a step.
e2e    = the same metric through the public API with Y copied from pinned host
         memory every step and the factors read back.
Prints one JSON line (rank 0).  Multi-GPU (torchrun) runs independent
replicas, one per rank (weak scaling); timing is the max over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "dense-tensor GB/s (sketch+core) vs HBM peak; FFCP time-to-fit vs plain FP32"
DEFAULT_CONFIG = "c4"
DEFAULT_PREC = "tc"
DEFAULT_SKETCH = "independent"
FALLBACK_HBM_GBS = 6800.0


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d.get("hbm_gbs", FALLBACK_HBM_GBS)), "measured"
    return FALLBACK_HBM_GBS, "fallback"


def _code_without_comments(src: str) -> str:
    """C++/CUDA source with its // and /* */ comments removed; string and
    character literals are kept whole.  An edit of a comment alone then
    leaves the kernel's hash unchanged."""
    out, i, n = [], 0, len(src)
    while i < n:
        c = src[i]
        if c in "\"'":
            j = i + 1
            while j < n and src[j] != c:
                j += 2 if src[j] == "\\" else 1
            out.append(src[i:j + 1])
            i = j + 1
        elif src.startswith("//", i):
            j = src.find("\n", i)
            i = n if j < 0 else j
        elif src.startswith("/*", i):
            j = src.find("*/", i + 2)
            i = n if j < 0 else j + 2
            out.append(" ")
        else:
            out.append(c)
            i += 1
    return "".join(out)


def _kernel_source_sha(prec: str) -> str:
    """Hash of the sketch kernel's code (comments excluded): the committed
    ncu traffic figure applies only while it matches."""
    return source_sha(["tc_sketch.cu", "tc_common.cuh"] if prec == "tc" else ["sketch_simt.cu"])


def source_sha(names) -> str:
    """First 16 hex digits of the SHA-256 of the named files under csrc/,
    comments removed, in the given order."""
    h = hashlib.sha256()
    for n in names:
        p = os.path.join(ROOT, "paper_1412_1885_gb300", "csrc", n)
        if os.path.exists(p):
            h.update(_code_without_comments(open(p, encoding="utf-8").read()).encode("utf-8"))
    return h.hexdigest()[:16]


def _traffic_from_profiles(kernel_tag: str, workload: str, sha: str):
    """Per-launch DRAM bytes of the sketch kernel from the committed ncu
    summary, if it was taken on the current kernel source."""
    p = os.path.join(ROOT, "profiles", f"{kernel_tag}_{workload}.md")
    if not os.path.exists(p):
        return None
    vals = {}
    for line in open(p):
        if ":" in line and line.strip().startswith("- "):
            k, v = line.strip()[2:].split(":", 1)
            vals[k.strip()] = v.strip()
    if vals.get("kernel_source_sha") != sha:
        return None
    try:
        return float(vals["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out = ""
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        sm.sort()
        med = sm[len(sm) // 2] if sm else None
        return {"sm_mhz": med, "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def max_over_ranks(x: float, pg, device) -> float:
    """The largest value of x over all ranks (the job's time is its slowest
    rank's); x itself without a process group."""
    if pg is None:
        return float(x)
    import torch

    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def job_value(alg_bytes_per_replica: int, world: int, ms: float) -> float:
    """Whole-job GB/s: every rank processes its own replica of the workload
    (weak scaling), timed by the slowest rank."""
    return world * alg_bytes_per_replica / (ms * 1e-3) / 1e9


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def cpu_oracle_sample(w, seconds_target=10.0, max_block=200_000_000, rule="ls"):
    """Time the FP64 oracle (as it stands) on a leading sub-block of the
    workload on the host cores: sketch + QR + core over the block, then ALS on
    its core.  A small block is timed first to size the measured block (at
    most `max_block` elements); the measured block is run repeatedly until
    about `seconds_target` seconds of oracle work have accumulated.
    Returns (GB/s of the block's two passes, description, seconds)."""
    import numpy as np

    import oracle
    import synth

    def block(n_target):
        shape = list(w.shape)
        sub = [min(s, max(r + w.p, 8)) for s, r in zip(shape, w.ranks)]
        for n in reversed(range(w.N)):
            while sub[n] < shape[n] and int(np.prod(sub)) * 2 <= n_target:
                sub[n] = min(shape[n], sub[n] * 2)
        return sub

    def prepare(sub):
        sw = synth.scaled(w, sub)
        return (sw, synth.host_tensor(sw), synth.sketch_matrices(sw.shape, sw.Rt, sw.seed),
                synth.init_factors(sw.Rt, sw.als_R, sw.seed),
                synth.init_factors(sw.shape, sw.als_R, sw.seed, dist="uniform") if sw.nonneg else None)

    def run(prep):
        sw, Y, W, B0, A0 = prep
        t0 = time.perf_counter()
        tk = oracle.rand_tucker(Y, W)
        if sw.nonneg:
            oracle.cp_als_nonneg(tk["G"], tk["U"], A0, max_sweeps=min(sw.als_max_sweeps, 200), tol=sw.als_tol,
                                 rule=rule)
        else:
            oracle.cp_als(tk["G"], B0, max_sweeps=min(sw.als_max_sweeps, 200), tol=sw.als_tol)
        return time.perf_counter() - t0

    probe = block(2_000_000)
    dt = run(prepare(probe))
    n_probe = int(np.prod(probe))
    sub = block(int(min(max_block, max(n_probe, n_probe * seconds_target / max(dt, 1e-3)))))
    prep = prepare(sub)
    total, reps = 0.0, 0
    while reps < 1 or (total < seconds_target and reps < 100):
        total += run(prep)
        reps += 1
    nbytes = 2 * w.itemsize * int(np.prod(sub)) * reps
    desc = (f"oracle rand_tucker + ALS (<=200 sweeps) on the leading {'x'.join(map(str, sub))} block "
            f"of {w.name}, {reps} run(s), {total:.1f} s")
    return nbytes / total / 1e9, desc, total


ONE_THREAD_ENV = {"OMP_NUM_THREADS": "1", "OPENBLAS_NUM_THREADS": "1", "MKL_NUM_THREADS": "1",
                  "NUMEXPR_NUM_THREADS": "1", "VECLIB_MAXIMUM_THREADS": "1"}


def cpu_oracle_one_thread(config: str, shape: str, rule: str, seconds: float = 6.0):
    """The same oracle sample on one host thread: a child process with the
    BLAS and OpenMP thread counts pinned to 1 (they are fixed when numpy
    loads).  Returns (GB/s, description) or (None, reason)."""
    cmd = [sys.executable, os.path.abspath(__file__), "--oracle-one-thread", "--config", config,
           "--nonneg-rule", rule, "--oracle-seconds", str(seconds)]
    if shape:
        cmd += ["--shape", shape]
    try:
        r = subprocess.run(cmd, capture_output=True, text=True, timeout=600, env=dict(os.environ, **ONE_THREAD_ENV))
        d = json.loads(r.stdout.strip().splitlines()[-1])
        return d["value"], d["sample"]
    except Exception as e:  # the all-core figure stands alone then
        return None, f"not measured: {type(e).__name__}"


def _fit_run(fn):
    """(device ms, result) of one call, CUDA events on the current stream."""
    import torch

    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    out = fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1), out


def compress_forms(t, ctx, w, Y, Wd, prec, dev, reps=2):
    """One-pass sketch + core, Alg. 2 (tucker_seq) and RandTucker2i (two
    tucker_refine passes from Gaussian factors, then the core) on the timed
    tensor: device ms per run (CUDA events, after a warm run), the passes
    over Y each makes, GB/s of Y read, and the relative reconstruction error
    sqrt(1 - ||G||^2 / ||Y||^2) (orthonormal factors)."""
    import math

    import torch

    import synth

    U0 = [torch.as_tensor(u, device=dev) for u in synth.random_factors(w.shape, w.Rt, w.seed)]

    def one_pass():
        nrm = torch.empty((), dtype=torch.float64, device=dev)
        U, _ = t.tucker_sketch(ctx, Y, Wd, w.ranks, w.p, prec, normY2=nrm)
        G, _ = t.tucker_core(ctx, Y, U, w.ranks, w.p, prec, want_norm=False)
        return G, nrm

    def seq():
        _, G, nrm = t.tucker_seq(ctx, Y, Wd, w.ranks, w.p, prec)
        return G, nrm

    def two_i():
        _, G, nrm = t.rand_tucker_2i(ctx, Y, U0, [w.seed + 101, w.seed + 102], w.ranks, w.p, prec)
        return G, nrm

    y_bytes = w.itemsize * w.numel
    out = {}
    for name, fn, passes in (("one_pass", one_pass, 2), ("alg2_sequential", seq, 2), ("randtucker2i", two_i, 5)):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            G, nrm = fn()
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        n2 = float(nrm.item())
        err = math.sqrt(max(0.0, n2 - float((G.double() ** 2).sum().item())) / n2)
        out[name] = {"ms": ms, "passes_over_Y": passes, "GBps_of_Y": passes * y_bytes / (ms * 1e-3) / 1e9,
                     "rel_error": err}
    out["note"] = ("device ms per run with Y resident; rel_error = ||Y - [[G; U]]|| / ||Y|| on the bench tensor "
                   "(CP model plus noise); RandTucker2i: two refinement passes from Gaussian factors, then the core")
    return out


def learned_setup(t, ctx, w, prec, n_train, n_eval, dev):
    """Learned-initialiser workload: build a training set with the method
    (compress, FFCP from the HOSVD start to convergence), train the MLP, then
    compare ALS from the random, HOSVD and learned starts on held-out tensors
    (sweeps, final fit, device time from the resident core to the factors).
    Everything here is set-up and evaluation, outside the timed steps."""
    import numpy as np
    import torch

    import synth
    from paper_1412_1885_gb300 import learned_init as li

    N, Rt, hidden = w.N, w.Rt[0], 1024
    m = t.Mlp(ctx, N, Rt, hidden, max_batch=256)
    m.set_params(synth.mlp_init_params(N, Rt, hidden, w.seed, hosvd_start=True, out_scale=0.1))

    def tensor(k, split):
        wk = synth.learned_init_workload(k, split, w.shape, Rt)
        Y, _ = synth.device_tensor(wk, device=dev)
        B0 = [torch.as_tensor(b, device=dev) for b in synth.init_factors(wk.Rt, wk.als_R, wk.seed)]
        return wk, Y, None, B0  # test matrices drawn inside the library from the workload's seed

    t0 = time.perf_counter()
    items = []
    for k in range(n_train):
        wk, Y, Wd, B0 = tensor(k, 1)
        it = li.method_sample(ctx, m, Y, Wd, list(wk.ranks), 0, wk.als_R, B0, prec=prec, init="hosvd",
                              max_sweeps=300, seed=synth.omega_seed(wk))
        items.append({kk: v for kk, v in it.items() if kk not in ("U", "Gc")})
        del Y
    data = li.stack(items)
    gen_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    hist = li.train(m, data, epochs=40, batch=128, lr=2e-4 if Rt > 12 else 1e-3, alpha=0.5)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    res = {k: {"sweeps": [], "fit": [], "ms": []} for k in ("random", "hosvd", "learned")}
    for k in range(n_eval):
        wk, Y, Wd, B0 = tensor(k, 2)
        nrm = torch.empty((), dtype=torch.float64, device=dev)
        U, _ = t.tucker_sketch(ctx, Y, Wd, list(wk.ranks), 0, prec, seed=synth.omega_seed(wk), normY2=nrm)
        G, _ = t.tucker_core(ctx, Y, U, list(wk.ranks), 0, prec, want_norm=False)
        args = (ctx, G, U, wk.shape, list(wk.ranks), 0, t._dtype_code(Y), wk.als_R, wk.als_max_sweeps, wk.als_tol)
        runs = {"random": lambda: t.ffcp_als(*args, B0=B0, normY2=nrm),
                "hosvd": lambda: t.ffcp_als(*args, init="hosvd", normY2=nrm),
                "learned": lambda: t.ffcp_als(*args, normY2=nrm, B0=m.predict_init(G, U, wk.shape, list(wk.ranks), 0,
                                                                                  t._dtype_code(Y), wk.als_R))}
        for name, fn in runs.items():
            ms, o = _fit_run(fn)
            res[name]["sweeps"].append(o["sweeps"])
            res[name]["fit"].append(o["fit_Y"])
            res[name]["ms"].append(ms)
        ms_p, _ = _fit_run(lambda: m.predict_init(G, U, wk.shape, list(wk.ranks), 0, t._dtype_code(Y), wk.als_R))
        res["learned"].setdefault("ms_predict", []).append(ms_p)
        del Y
    ev = {k: {"sweeps_median": float(np.median(v["sweeps"])), "sweeps_mean": float(np.mean(v["sweeps"])),
              "sweeps_p90": float(np.percentile(v["sweeps"], 90)), "ms_median": float(np.median(v["ms"])),
              "ms_mean": float(np.mean(v["ms"])), "fit_Y_mean": float(np.mean(v["fit"])),
              **({"ms_predict_median": float(np.median(v["ms_predict"]))} if "ms_predict" in v else {})}
          for k, v in res.items()}
    info = {"train_tensors": int(data.G.shape[0]), "generated": n_train, "epochs": 40, "hidden": hidden,
            "loss_first_epoch": hist[0], "loss_last_epoch": hist[-1], "loss_best_epoch": min(hist),
            "loss_per_epoch": hist, "grad_clip": 1.0, "gen_s": gen_s, "train_s": train_s,
            "eval_tensors": n_eval, "eval": ev}
    return m, info


def run_reference(args, w):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    import numpy as np  # noqa: F401

    cores = os.cpu_count()
    vals = []
    desc = ""
    for i in range(args.warmup + args.steps):
        v, desc, _ = cpu_oracle_sample(w, rule=args.nonneg_rule)
        if i >= args.warmup:
            vals.append(v)
    vals.sort()
    v = vals[len(vals) // 2]
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "GB/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": None, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w.name, "shape": list(w.shape), "ranks": list(w.ranks), "p": w.p,
                       "R": w.als_R},
            "cpu_baseline": {"value": v, "unit": "GB/s", "cores": cores, "kind": "oracle", "sample": desc},
            "e2e": {"value": v, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--config", default=DEFAULT_CONFIG)
    ap.add_argument("--prec", default=DEFAULT_PREC, choices=["tc", "simt"])
    ap.add_argument("--shape", default="", help="comma-separated dims replacing the workload's shape")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--no-ttf", action="store_true", help="skip the time-to-fit comparison of the forms")
    ap.add_argument("--no-forms", action="store_true",
                    help="skip the comparison of the one-pass, sequential (Alg. 2) and RandTucker2i compressions")
    ap.add_argument("--train", type=int, default=2048, help="learned-init workload: training tensors")
    ap.add_argument("--eval", type=int, default=64, help="learned-init workload: held-out tensors")
    ap.add_argument("--nonneg-rule", default="ls", choices=["ls", "hals", "mu"],
                    help="update rule of the nonnegative workloads: projected LS, HALS (Eq. 8), MU (Eq. 15)")
    ap.add_argument("--sketch", default=DEFAULT_SKETCH, choices=["shared", "independent"],
                    help="sketch family: Khatri-Rao factors shared between the modes, or drawn per mode")
    ap.add_argument("--oracle-one-thread", action="store_true", help=argparse.SUPPRESS)
    ap.add_argument("--oracle-seconds", type=float, default=10.0, help=argparse.SUPPRESS)
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3

    import synth

    w = synth.WORKLOADS[args.config]
    if args.shape:
        # same data model, ranks and dtype at another size (small ncu captures)
        w = synth.scaled(w, [int(x) for x in args.shape.split(",")])
    if args.oracle_one_thread:
        v, desc, _ = cpu_oracle_sample(w, seconds_target=args.oracle_seconds, rule=args.nonneg_rule)
        print(json.dumps({"value": v, "sample": desc}), flush=True)
        return 0
    if args.impl == "reference":
        return run_reference(args, w)

    import numpy as np
    import torch

    import paper_1412_1885_gb300 as t
    from paper_1412_1885_gb300 import build

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dev = f"cuda:{local}"
    pg = None
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device(dev))
        pg = dist
    if rank == 0:
        build.build()
    if pg:
        pg.barrier()
    t.lib()

    # ---- inputs (untimed): Y generated in HBM, W / init from the seeded generators
    ctx = t.Context(local)
    model, li_info = None, None
    if args.config == "c5":
        model, li_info = learned_setup(t, ctx, w, args.prec, args.train, args.eval, dev)
        # the timed tensor: held-out tensor 0 of the learned-initialiser workload
        w = synth.learned_init_workload(0, 2, w.shape, w.Rt[0])
    Y, A_true = synth.device_tensor(w, device=dev)
    W = synth.sketch_matrices(w.shape, w.Rt, w.seed, shared=args.sketch == "shared")
    Wd = synth.device_sketch(W, dev)
    B0 = [torch.as_tensor(b, device=dev) for b in synth.init_factors(w.Rt, w.als_R, w.seed)]
    A0 = [torch.as_tensor(a, device=dev) for a in synth.init_factors(w.shape, w.als_R, w.seed, dist="uniform")]
    torch.cuda.synchronize()

    def step(Yin, Ydev=None, prec=args.prec):
        return t.decompose(ctx, Yin, Wd, w.ranks, w.p, w.als_R, prec, nonneg=args.nonneg_rule if w.nonneg else False,
                           Y_dev=Ydev,
                           max_sweeps=w.als_max_sweeps, tol=w.als_tol, B0=None if w.nonneg else B0,
                           A0=A0 if w.nonneg else None, check_every=16, model=model)

    for _ in range(args.warmup):
        out = step(Y)
    torch.cuda.synchronize()

    # ---- timed region (device time, CUDA events on the current stream)
    sampler = ClockSampler(local)
    ctx.profile(True)
    l0 = ctx.launch_count()
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    sampler.start()
    time.sleep(0.3)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    sweeps = []
    for _ in range(args.steps):
        out = step(Y)
        sweeps.append(out["sweeps"])
    e1.record()
    torch.cuda.synchronize()
    clocks = sampler.stop()
    if pg:
        pg.barrier()
    ms = e0.elapsed_time(e1) / args.steps
    launches = ctx.launch_count() - l0
    sk_ms, sk_n = ctx.profile_read(0)
    co_ms, co_n = ctx.profile_read(1)
    ctx.profile(False)
    ms = max_over_ranks(ms, pg, dev)
    y_bytes = w.itemsize * w.numel
    alg_bytes = 2 * y_bytes
    value = job_value(alg_bytes, ws, ms)

    # ---- end to end: Y from pinned host memory each step, factors read back
    e2e = None
    if not args.no_e2e:
        Yh = torch.empty(Y.shape, dtype=Y.dtype, pin_memory=True)
        Yh.copy_(Y)
        torch.cuda.synchronize()
        h2d = Yh.numel() * Yh.element_size()
        d2h = 0
        if pg:
            pg.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            # the public call on host data: Y crosses the link inside decompose (tdk_copy_in)
            o = step(Yh, Y)
            host = [t.copy_out(ctx, a) for a in o["A"]]
            d2h = sum(a.numel() * a.element_size() for a in host)
        torch.cuda.synchronize()
        dt = max_over_ranks((time.perf_counter() - t0) / args.e2e_steps, pg, dev)
        e2e = {"value": job_value(alg_bytes, ws, dt * 1e3), "unit": "GB/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "ms_per_step": dt * 1e3}
        del Yh

    # ---- FFCP time-to-fit: this form vs the plain CUDA-core form, same tensor
    ttf = None
    if not args.no_ttf and rank == 0:
        forms = {}
        for form in dict.fromkeys([args.prec, "simt"]):
            step(Y, prec=form)  # warm this form's kernels
            ms_f, o = _fit_run(lambda: step(Y, prec=form))
            forms[form] = {"ms": ms_f, "fit_Y": o["fit_Y"], "sweeps": o["sweeps"]}
        ttf = {"forms": forms, "note": "device ms from Y resident in HBM to the factors A_n, one run per form; "
                                       "simt = the plain CUDA-core form (FP32 arithmetic for FP32/BF16 data)"}
        if "simt" in forms and args.prec in forms and args.prec != "simt":
            ttf["speedup_vs_simt"] = forms["simt"]["ms"] / forms[args.prec]["ms"]
            ttf["fit_Y_diff"] = abs(forms["simt"]["fit_Y"] - forms[args.prec]["fit_Y"])

    # ---- the three compressions of Sec. IV-A on the same tensor: passes over
    # Y, device time and reconstruction error ||Y - [[G; U]]|| / ||Y||
    forms = None
    if not args.no_forms and rank == 0:
        forms = compress_forms(t, ctx, w, Y, Wd, args.prec, dev)

    peak, peak_kind = _peaks()
    sk_avg = sk_ms / max(sk_n, 1)
    achieved = y_bytes / (sk_avg * 1e-3) / 1e9 if sk_n else None
    sha = _kernel_source_sha(args.prec)
    kernel_tag = "tc_sketch" if args.prec == "tc" else "sketch_simt"
    roofline = {"bound": "hbm", "kernel": kernel_tag, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": (achieved / peak) if achieved else None, "peak_kind": peak_kind,
                "traffic": _traffic_from_profiles(kernel_tag, args.config, sha),
                "algorithmic_bytes_per_launch": y_bytes, "avg_launch_ms": sk_avg,
                "kernel_source_sha": sha,
                "core_pass": {"achieved": (y_bytes / (co_ms / max(co_n, 1) * 1e-3) / 1e9) if co_n else None,
                              "avg_launch_ms": co_ms / max(co_n, 1)}}
    cpu = None
    if rank == 0 and not args.no_cpu:
        cv, cdesc, _ = cpu_oracle_sample(w, rule=args.nonneg_rule)
        v1, d1 = cpu_oracle_one_thread(args.config, args.shape, args.nonneg_rule)
        cpu = {"value": cv, "unit": "GB/s", "cores": os.cpu_count(), "kind": "oracle", "sample": cdesc,
               "one_thread": {"value": v1, "unit": "GB/s", "cores": 1, "sample": d1}}
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": {"f64": "f64", "f32": "f32", "bf16": "bf16"}[w.dtype],
                "data": "synthetic",
                "config": {"workload": w.name, "shape": list(w.shape), "ranks": list(w.ranks), "p": w.p,
                           "R": w.als_R, "prec": args.prec, "nonneg": w.nonneg,
                           "nonneg_rule": args.nonneg_rule if w.nonneg else None, "sketch": args.sketch,
                           "l2": "inputs larger than L2 (no flush)",
                           "parallelism": f"replicas{ws}" if ws > 1 else "single"},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks,
                "gpu_launches": launches,
                "als": {"sweeps": sweeps, "fit_core": out["fit_core"], "fit_Y": out["fit_Y"],
                        "ms_last": out["ms"]},
                "sketch_ms": sk_avg, "core_ms": co_ms / max(co_n, 1), "time_to_fit": ttf,
                "compress_forms": forms}
        if li_info is not None:
            line["learned_init"] = li_info
            line["config"]["train_tensors"] = li_info["train_tensors"]
        print(json.dumps(line), flush=True)
    ctx.close()
    if pg:
        pg.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
