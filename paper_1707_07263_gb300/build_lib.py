"""Builds ``libgbfft.so`` in-tree from ``csrc/*.cu`` with nvcc for sm_103a.

Each translation unit is compiled in parallel; the shared library links the
CUDA runtime statically so it loads without extra library paths.

Beside it, the same objects with the planner sources recompiled under
``-DGBFFT_TEST_HOOKS`` are linked into ``libgbfft_testhooks.so``, a test-only
library in which environment variables force planner choices (passes,
splits, staging kernels, tile sizes) and plant a missing producer in an
uneven-batch plan (the bounded-wait timeout test).  The product library reads
no environment variable.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libgbfft.so")
TEST_LIB = os.path.join(HERE, "libgbfft_testhooks.so")
TEST_SRCS = ("many.cu", "mixed.cu", "plan.cu")   # the sources whose test build differs
TEST_FLAGS = ["-DGBFFT_TEST_HOOKS"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden",
         "--expt-relaxed-constexpr"]


def nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libgbfft.so")
    return cand


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return (glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h"))
            + [os.path.join(HERE, "..", "include", "gbfft.h"), os.path.abspath(__file__)])


def _compile(src: str, obj: str, extra) -> str:
    cmd = [nvcc(), *ARCH, *FLAGS, *extra, "-I", os.path.join(HERE, "..", "include"), "-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {os.path.basename(src)}:\n{r.stdout}\n{r.stderr}")
    return r.stderr


def _link(out: str, objs) -> None:
    tmp = out + f".tmp{os.getpid()}"
    cmd = [nvcc(), *ARCH, "-shared", "-cudart", "static", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, out)


def build(force: bool = False, verbose: bool = False, extra=()) -> str:
    os.makedirs(BUILD, exist_ok=True)
    srcs = _sources()
    dep_mtime = max(os.path.getmtime(p) for p in _deps())

    def obj(src, test=False):
        return os.path.join(BUILD, os.path.basename(src)[:-3] + ("_testhooks.o" if test else ".o"))

    units = [(s, obj(s), list(extra)) for s in srcs]
    units += [(os.path.join(CSRC, t), obj(t, True), list(extra) + TEST_FLAGS) for t in TEST_SRCS]
    jobs = []
    for s, o, flags in units:
        if force or not os.path.exists(o) or os.path.getmtime(o) < max(os.path.getmtime(s), dep_mtime):
            jobs.append((s, o, flags))
    if jobs:
        workers = min(len(jobs), max(1, os.cpu_count() or 1))
        with cf.ThreadPoolExecutor(max_workers=workers) as ex:
            futs = {ex.submit(_compile, s, o, flags): s for s, o, flags in jobs}
            for f in cf.as_completed(futs):
                msg = f.result()
                if verbose and msg:
                    sys.stderr.write(msg)
    objs = [obj(s) for s in srcs]
    if force or jobs or not os.path.exists(LIB):
        _link(LIB, objs)
    if force or jobs or not os.path.exists(TEST_LIB):
        _link(TEST_LIB, [obj(s, os.path.basename(s) in TEST_SRCS) for s in srcs])
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
