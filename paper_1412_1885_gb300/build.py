"""Build libtdk.so in-tree for sm_103a (nvcc, one object per translation unit,
compiled in parallel, linked as a shared library with the static CUDA runtime).

Beside it, libtdk_test.so: the same sources compiled with -DTDK_TESTING (the
test hooks: a forced workspace-allocation failure, a device wait that nothing
satisfies, raw kernel calls, cycle-counter profiling switches) and
-DTDK_CHECKED (bounds checks on the kernels' index computations that report
through the status word instead of faulting).  The product library exports
none of the hooks and carries none of the checks."""
from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libtdk.so")
TEST_LIB = os.path.join(HERE, "libtdk_test.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr"]
LINK = ["-lcudart_static", "-ldl", "-lrt", "-lpthread"]


def _nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.sep not in c or os.path.exists(c)):
            return c
    return "nvcc"


def sources():
    return sorted(f for f in os.listdir(CSRC) if f.endswith(".cu"))


def _deps_mtime() -> float:
    t = os.path.getmtime(os.path.abspath(__file__))
    for d in (CSRC, os.path.join(HERE, "..", "include")):
        for f in os.listdir(d):
            t = max(t, os.path.getmtime(os.path.join(d, f)))
    return t


def build(force: bool = False, verbose: bool = False, extra=()) -> str:
    dep = _deps_mtime()
    if (not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= dep and os.path.exists(TEST_LIB)
            and os.path.getmtime(TEST_LIB) >= dep):
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()

    def one(job):
        src, testing = job
        obj = os.path.join(BUILD, src[:-3] + (".test.o" if testing else ".o"))
        cmd = [nvcc, *ARCH, *FLAGS, *extra, *(["-DTDK_TESTING", "-DTDK_CHECKED"] if testing else []), "-c",
               os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            print(r.stdout + r.stderr, file=sys.stderr)
        return obj

    srcs = sources()
    jobs = [(s, False) for s in srcs] + [(s, True) for s in srcs]
    with cf.ThreadPoolExecutor(max_workers=min(24, os.cpu_count() or 4)) as ex:
        objs = dict(zip(jobs, ex.map(one, jobs)))
    for path, testing in ((LIB, False), (TEST_LIB, True)):
        parts = [objs[(s, testing)] for s in srcs]
        tmp = path + ".tmp"
        r = subprocess.run([nvcc, *ARCH, "-shared", "-o", tmp, *parts, *LINK], capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, path)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
