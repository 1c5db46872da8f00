"""Build libtbsma.so in-tree with nvcc for sm_103a (B300)."""

from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = os.path.join(HERE, "csrc", "tbsma.cu")
DEPS = [os.path.join(HERE, "csrc", f) for f in ("device.cuh", "nlist.cuh", "pair.cuh", "md.cuh", "persist.cuh", "topo.cuh")]
HEADER = os.path.join(ROOT, "include", "tbsma.h")
LIB = os.path.join(HERE, "libtbsma.so")

NVCC_FLAGS = [
    "-O3",
    "-std=c++17",
    "-gencode",
    "arch=compute_103a,code=sm_103a",
    "-lineinfo",
    "-Xcompiler",
    "-fPIC",
    "-shared",
]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.isabs(cand) and os.path.exists(cand) or not os.path.isabs(cand)):
            return cand
    return "nvcc"


def stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(p) > t for p in [SRC, HEADER, *DEPS])


def build(force: bool = False, verbose: bool = False, extra: list[str] | None = None) -> str:
    if force or stale():
        cmd = [nvcc(), *NVCC_FLAGS, *(extra or []), "-I", os.path.join(ROOT, "include"),
               "-o", LIB, SRC]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        subprocess.run(cmd, check=True)
    return LIB


if __name__ == "__main__":
    build(force=True, verbose=True, extra=sys.argv[1:])
