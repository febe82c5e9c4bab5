"""Build of the in-tree CUDA libraries for sm_103a.

``_build/libhpeel.so``: each ``csrc/*.cu`` file is compiled by nvcc in
parallel into an object, then the objects are linked into one shared library
(CUDA runtime linked statically, so it loads beside any PyTorch build).
``_build/libhpeel_measure.so``: the benchmark's measurement probe
(``measure/*.cu``), kept out of the peeling library.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libhpeel.so")
MEASURE = os.path.join(HERE, "measure")
MEASURE_LIB = os.path.join(BUILD, "libhpeel_measure.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2",
         "--expt-relaxed-constexpr", "-I", INCLUDE, "-I", CSRC]


def nvcc() -> str:
    path = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(path):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libhpeel")
    return path


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _measure_sources():
    return sorted(glob.glob(os.path.join(MEASURE, "*.cu")))


def _deps():
    return (_sources() + _measure_sources() + glob.glob(os.path.join(CSRC, "*.cuh"))
            + glob.glob(os.path.join(MEASURE, "*.h")) + [os.path.join(INCLUDE, "hpeel.h")])


def up_to_date() -> bool:
    if not (os.path.exists(LIB) and os.path.exists(MEASURE_LIB)):
        return False
    t = min(os.path.getmtime(LIB), os.path.getmtime(MEASURE_LIB))
    return all(os.path.getmtime(p) <= t for p in _deps())


def build(force: bool = False, verbose: bool = False, extra=()) -> str:
    if not force and up_to_date():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    cc = nvcc()
    objs = []

    def compile_one(src):
        prefix = "measure_" if os.path.dirname(src) == MEASURE else ""
        obj = os.path.join(BUILD, prefix + os.path.basename(src)[:-3] + ".o")
        cmd = [cc, *ARCH, *FLAGS, "-I", MEASURE, *extra, "-c", src, "-o", obj]
        if verbose:
            print(" ".join(cmd))
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            print(r.stdout, r.stderr)
        return obj

    srcs = _sources()
    msrcs = _measure_sources()
    with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 4)) as ex:
        objs = list(ex.map(compile_one, srcs + msrcs))
    for out, group in ((LIB, objs[:len(srcs)]), (MEASURE_LIB, objs[len(srcs):])):
        tmp = out + f".tmp{os.getpid()}"
        cmd = [cc, *ARCH, "-shared", "-o", tmp, *group]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link of {out} failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, out)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv,
                extra=["-Xptxas", "-v"] if "--ptxas" in sys.argv else ()))
