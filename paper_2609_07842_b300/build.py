"""Build libvbc.so in-tree with nvcc for sm_103a (B300).

    python -m paper_2609_07842_b300.build

The library is built from csrc/vbc_api.cu (runtime, C ABI and, through its
includes, the kernels) and csrc/vbc_noalloc.cu (the allocation-free
evaluation); the C ABI it exports is declared in include/vbc.h.
"""
from __future__ import annotations

import glob
import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
SRCS = [os.path.join(PKG, "csrc", f) for f in ("vbc_api.cu", "vbc_noalloc.cu", "vbc_serve.cpp")]
# every source and header of the library: a change to any of them rebuilds it
DEPS = sorted(glob.glob(os.path.join(PKG, "csrc", "*.cu")) + glob.glob(os.path.join(PKG, "csrc", "*.cuh")) +
              glob.glob(os.path.join(PKG, "csrc", "*.cpp")) + glob.glob(os.path.join(ROOT, "include", "*.h")))
LIB = os.path.join(PKG, "libvbc.so")

NVCC_FLAGS = [
    "-O3", "-std=c++17",
    "-gencode", "arch=compute_103a,code=sm_103a",
    "-lineinfo",
    "-Xcompiler", "-fPIC", "-shared",
]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile the library if it is missing or older than its sources; returns its path."""
    stale = force or not os.path.exists(LIB) or any(
        os.path.getmtime(d) > os.path.getmtime(LIB) for d in DEPS)
    if stale:
        tmp = LIB + ".tmp%d" % os.getpid()
        cmd = [nvcc(), *NVCC_FLAGS, "-I" + os.path.join(ROOT, "include"), "-o", tmp, *SRCS]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
            print(" ".join(cmd), file=sys.stderr)
        subprocess.run(cmd, check=True)
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
