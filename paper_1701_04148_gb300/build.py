"""Build the in-tree CUDA libraries for sm_103a (nvcc, no cmake): libsfgb300.so (the sketch
library, csrc/*.cu) and libsfbench.so (the measurement kernels of the benchmark and the bounded-wait
failure test, csrc/bench/*.cu).

Each translation unit compiles in parallel (`nvcc -c`), then one `nvcc -shared` per library links
them.  The results land in paper_1701_04148_gb300/_build/ (git-ignored).  Usage:
    python -m paper_1701_04148_gb300.build [--force] [--verbose]
"""
from __future__ import annotations

import argparse
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libsfgb300.so")
BENCH_LIB = os.path.join(BUILD, "libsfbench.so")
BENCH_SRC = os.path.join(CSRC, "bench")
ROOT = os.path.dirname(HERE)
INCLUDE = os.path.join(ROOT, "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2", "-Xcompiler", "-pthread",
              "--expt-relaxed-constexpr", "-I" + INCLUDE, "-I" + CSRC]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found: the SF-sketch CUDA library cannot be built")


def sources(folder: str = CSRC) -> list[str]:
    return sorted(os.path.join(folder, f) for f in os.listdir(folder) if f.endswith(".cu"))


def _deps() -> list[str]:
    out = []
    for d in (CSRC, BENCH_SRC, INCLUDE):
        for f in os.listdir(d):
            if f.endswith((".cu", ".cuh", ".h")):
                out.append(os.path.join(d, f))
    return out


def up_to_date() -> bool:
    if not os.path.exists(LIB) or not os.path.exists(BENCH_LIB):
        return False
    t = min(os.path.getmtime(LIB), os.path.getmtime(BENCH_LIB))
    return all(os.path.getmtime(p) <= t for p in _deps() + [__file__])


def build(force: bool = False, verbose: bool = False, extra_flags: list[str] | None = None) -> str:
    if not force and up_to_date():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    nv = nvcc()
    flags = NVCC_FLAGS + (extra_flags or [])

    def compile_one(src: str) -> str:
        sub = "bench_" if os.path.dirname(src) == BENCH_SRC else ""
        obj = os.path.join(BUILD, sub + os.path.basename(src).replace(".cu", ".o"))
        cmd = [nv] + ARCH + flags + ["-c", src, "-o", obj]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {os.path.basename(src)}:\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            sys.stderr.write(r.stdout + r.stderr)
        return obj

    srcs, bsrcs = sources(), sources(BENCH_SRC)
    with cf.ThreadPoolExecutor(max_workers=min(8, len(srcs) + len(bsrcs))) as ex:
        objs = list(ex.map(compile_one, srcs + bsrcs))
    for lib, part in ((LIB, objs[:len(srcs)]), (BENCH_LIB, objs[len(srcs):])):
        tmp = lib + f".tmp{os.getpid()}"
        r = subprocess.run([nv] + ARCH + ["-shared", "-Xcompiler", "-pthread", "-o", tmp] + part, capture_output=True,
                           text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, lib)
    return LIB


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("--force", action="store_true")
    ap.add_argument("--verbose", action="store_true")
    a = ap.parse_args()
    print(build(force=a.force, verbose=a.verbose))
