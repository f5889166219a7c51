"""Build libsph.so in-tree with nvcc for sm_103a (B300).

Usage: python -m paper_2606_23891_b300.build [--force] [--check]

--check builds libsph_check.so instead: the same library compiled with
-DSPH_CHECK, whose kernels check every gathered and scattered index against
its buffer and report a violation as SPH_EBOUNDS (sph.py loads it when
SPH_CHECKED_BUILD=1).
"""
from __future__ import annotations

import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libsph.so")
LIB_CHECK = os.path.join(HERE, "libsph_check.so")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
         "-Xcompiler", "-Wall", "-Xcompiler", "-fopenmp", "-I" + os.path.join(ROOT, "include"),
         "-I" + CSRC, "--expt-relaxed-constexpr"]


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")) +
                  glob.glob(os.path.join(CSRC, "*.cpp")))


def inputs():
    return sources() + sorted(glob.glob(os.path.join(CSRC, "*.h")) +
                              glob.glob(os.path.join(CSRC, "*.cuh"))) + \
        [os.path.join(ROOT, "include", "sph.h"), os.path.abspath(__file__)]


def stale(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(p) > t for p in inputs())


def build(force: bool = False, verbose: bool = False, extra=(), check: bool = False) -> str:
    LIB = LIB_CHECK if check else globals()["LIB"]
    if check:
        extra = list(extra) + ["-DSPH_CHECK"]
    if not force and not stale(LIB):
        return LIB
    objdir = os.path.join(HERE, "_build_check" if check else "_build")
    os.makedirs(objdir, exist_ok=True)
    objs = []
    for src in sources():
        obj = os.path.join(objdir, os.path.basename(src) + ".o")
        cmd = [NVCC] + ARCH + FLAGS + list(extra) + ["-c", src, "-o", obj]
        if src.endswith(".cpp"):
            cmd = [NVCC] + FLAGS + list(extra) + ["-x", "c++", "-c", src, "-o", obj]
        if verbose:
            print(" ".join(cmd))
        subprocess.check_call(cmd)
        objs.append(obj)
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = [NVCC] + ARCH + ["-shared", "-Xcompiler", "-fopenmp", "-o", tmp] + objs + ["-lgomp"]
    subprocess.check_call(cmd)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True,
                extra=["-Xptxas", "-v"] if "--ptxas" in sys.argv else [],
                check="--check" in sys.argv))
