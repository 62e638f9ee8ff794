"""Build ``libfstat.so`` in-tree for sm_103a.

Each FFT-pass instantiation (precision x factor length) is its own object so
that nvcc runs in parallel; the objects are linked into one shared library
next to this file.  Run ``python -m paper_0912_4255_gb300.build`` or call
``build()``.
"""
from __future__ import annotations

import hashlib
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OBJ = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libfstat.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         "--expt-relaxed-constexpr", "-Xptxas", "-warn-spills"]
LOGS = range(6, 13)


def nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libfstat")
    return cand


def units():
    """(object name, source, extra defines)"""
    out = [("api", "api.cu", []), ("timemap", "timemap.cu", []),
           ("resample", "resample.cu", []), ("dispatch", "dispatch.cu", []),
           ("grad", "grad.cu", []), ("persist", "persist.cu", []),
           ("noalloc", "noalloc.cu", []), ("topk", "topk.cu", []),
           ("inject", "inject.cu", []), ("frontend", "frontend.cu", []),
           ("demod", "demod.cu", []),
           ("selftest", "selftest.cu", []), ("stats", "stats.cu", [])]
    for real in ("float", "double"):
        for L in LOGS:
            out.append((f"cols_{real}_{L}", "cols.cu", [f"-DFS_REAL={real}", f"-DFS_L1={L}"]))
            out.append((f"rows_{real}_{L}", "rows.cu", [f"-DFS_REAL={real}", f"-DFS_L2={L}"]))
    return [u for u in out if os.path.exists(os.path.join(CSRC, u[1]))]


def _sources_digest() -> str:
    h = hashlib.sha256()
    inc = os.path.join(os.path.dirname(HERE), "include", "fstat.h")
    for p in sorted(os.listdir(CSRC)) + [inc]:
        fp = p if os.path.isabs(p) else os.path.join(CSRC, p)
        if os.path.isfile(fp):
            with open(fp, "rb") as f:
                h.update(os.path.relpath(fp, os.path.dirname(HERE)).encode())   # same on every machine
                h.update(f.read())
    h.update(" ".join(ARCH + FLAGS).encode())
    return h.hexdigest()


# sources that compile or sequence the kernels of fstat_compute (time map,
# resampler, A/B/C reduction, both FFT passes); other entry points (top-k,
# injection, gradient, persistent and allocation-free modes) live elsewhere
PATH_SOURCES = ("fstat_internal.cuh", "passes.cuh", "timemap.cu", "resample.cu", "cols.cu", "rows.cu",
                "api.cu", "dispatch.cu")


def path_digest() -> str:
    """Digest of the fstat_compute kernels' sources and build flags: profile
    summaries quote it so that a reader (and bench.py) can tell whether the
    counters still describe the built kernels."""
    h = hashlib.sha256()
    inc = os.path.join(os.path.dirname(HERE), "include", "fstat.h")
    for name in PATH_SOURCES + (inc,):
        fp = os.path.join(CSRC, name)        # an absolute name stays as it is
        with open(fp, "rb") as f:
            h.update(os.path.basename(name).encode())
            h.update(f.read())
    h.update(" ".join(ARCH + FLAGS).encode())
    return h.hexdigest()


def build(jobs: int | None = None, verbose: bool = False, force: bool = False) -> str:
    """Compile every unit and link libfstat.so; returns the library path."""
    os.makedirs(OBJ, exist_ok=True)
    digest = _sources_digest()
    stamp = os.path.join(OBJ, "stamp")
    if not force and os.path.exists(LIB) and os.path.exists(stamp):
        with open(stamp) as f:
            if f.read().strip() == digest:
                return LIB
    cc = nvcc()
    jobs = jobs or max(1, min(32, os.cpu_count() or 1))

    def compile_one(u):
        name, src, defs = u
        obj = os.path.join(OBJ, name + ".o")
        cmd = [cc, *ARCH, *FLAGS, *defs, "-I", os.path.dirname(HERE), "-c",
               os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {name}:\n{r.stderr[-6000:]}")
        if verbose and r.stderr.strip():
            sys.stderr.write(f"[{name}] {r.stderr}\n")
        return obj

    us = units()
    with ThreadPoolExecutor(jobs) as ex:
        objs = list(ex.map(compile_one, us))
    tmp = LIB + ".tmp"
    r = subprocess.run([cc, *ARCH, "-shared", "-o", tmp, *objs], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr[-6000:]}")
    os.replace(tmp, LIB)
    with open(stamp, "w") as f:
        f.write(digest)
    return LIB


if __name__ == "__main__":
    import time
    t0 = time.time()
    print(build(verbose="-v" in sys.argv, force="-f" in sys.argv), f"{time.time() - t0:.1f}s")
