"""Compile the CUDA library libgid.so in-tree for sm_103a (B300).

Run as ``python -m paper_1908_01961_b300.build`` or call ``build()``.  nvcc
cross-compiles without a GPU.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libgid.so")
SOURCES = ["gid.cu", "gid_noalloc.cu", "gid_net.cu", "gid_cluster.cu"]
HEADERS = ["gid_kernels.cuh", "gid_net_kernels.cuh", "gid_net_internal.h", "gid_nvtx.h"]
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-lineinfo", "-std=c++17",
         "-Xcompiler", "-fPIC", "-shared", "--expt-relaxed-constexpr"]


def _inputs():
    return [os.path.join(CSRC, f) for f in SOURCES + HEADERS] + [os.path.join(ROOT, "include", "gid.h")]


def build(force: bool = False, verbose: bool = False, extra=()) -> str:
    """Build libgid.so if any source is newer than it; returns its path."""
    if not force and os.path.exists(LIB):
        t = os.path.getmtime(LIB)
        if all(os.path.getmtime(f) <= t for f in _inputs()):
            return LIB
    tmp = LIB + f".{os.getpid()}.tmp"
    cmd = [NVCC] + FLAGS + list(extra) + ["-I", os.path.join(ROOT, "include"), "-o", tmp] + \
        [os.path.join(CSRC, f) for f in SOURCES]
    if verbose:
        print(" ".join(cmd), file=sys.stderr)
    subprocess.check_call(cmd)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True, extra=["-Xptxas", "-v"] if "--ptxas" in sys.argv else [])
    print(LIB)
