"""Build step of the CUDA library: nvcc -> libccfr.so for sm_103a, in-tree.

Run ``python -m paper_2607_26901_b300.build_lib`` (or call ``build()``).  The
library is compiled without fast-math so that the binary32 candidate predicate
and the IEEE divisions and square roots match their definitions.
"""
from __future__ import annotations

import os
import subprocess
import sys
from pathlib import Path

PKG = Path(__file__).resolve().parent
CSRC = PKG / "csrc"
INCLUDE = PKG.parent / "include"
LIB = PKG / "_lib" / "libccfr.so"
SOURCES = ["ccfr_kernels.cu", "ccfr_api.cu", "ccfr_server.cpp"]
DEPS = SOURCES + ["ccfr_device.cuh", "ccfr_internal.h", "ccfr_df.cuh"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.sep not in c or Path(c).exists()):
            return c
    return "nvcc"


def stale() -> bool:
    if not LIB.exists():
        return True
    t = LIB.stat().st_mtime
    srcs = [CSRC / f for f in DEPS] + [INCLUDE / "ccfr.h"]
    return any(p.stat().st_mtime > t for p in srcs)


def build(force: bool = False, verbose: bool = False) -> Path:
    if not force and not stale():
        return LIB
    LIB.parent.mkdir(parents=True, exist_ok=True)
    tmp = LIB.with_suffix(f".{os.getpid()}.tmp")
    cmd = [nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-shared",
           "-I", str(INCLUDE), "-o", str(tmp)] + [str(CSRC / f) for f in SOURCES]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
        print(" ".join(cmd))
    subprocess.check_call(cmd)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
