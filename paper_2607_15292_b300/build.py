"""Builds libgcqbem.so in-tree for B300 (sm_103a) with nvcc.

    python paper_2607_15292_b300/build.py [--ptxas-v]

Run as a script (not through the package, whose import loads the library).

The library is plain C ABI (include/gcqbem.h); no PyTorch headers are used.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libgcqbem.so")
SOURCES = ["host.cpp", "gcqbem.cu", "apply_tc.cu", "peaks.cu"]
DEPS = ["internal.h", "opdata.h", "entry.cuh", "entryf.cuh", "tma.cuh", "tc.cuh", "aca3d.cuh", "faceaca.cuh",
        "apply.cuh", "solve.cuh", "receiver.cuh", "rkcq.cuh", "persist.cuh"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.isabs(cand) and os.path.exists(cand) or not os.path.isabs(cand)):
            return cand
    return "nvcc"


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    files = [os.path.join(CSRC, f) for f in SOURCES + DEPS] + [os.path.join(ROOT, "include", "gcqbem.h")]
    return any(os.path.getmtime(f) > t for f in files)


def build(force: bool = False, ptxas_verbose: bool = False) -> str:
    """Compiles every source to an object in parallel (one nvcc per
    translation unit), then links the shared library."""
    if not force and not _stale():
        return LIB
    objdir = os.path.join(HERE, "_build")
    os.makedirs(objdir, exist_ok=True)
    common = ["-O3", "-std=c++17", "-lineinfo", *ARCH, "-Xcompiler", "-fPIC,-O3", "-I", os.path.join(ROOT, "include"),
              "-I", CSRC, "--expt-relaxed-constexpr"]
    if ptxas_verbose:
        common = ["-Xptxas", "-v"] + common
    procs, objs = [], []
    for f in SOURCES:
        obj = os.path.join(objdir, os.path.splitext(f)[0] + ".o")
        objs.append(obj)
        procs.append(subprocess.Popen([nvcc(), *common, "-c", os.path.join(CSRC, f), "-o", obj]))
    bad = [f for f, p in zip(SOURCES, procs) if p.wait() != 0]
    if bad:
        raise RuntimeError(f"nvcc failed on {bad}")
    subprocess.run([nvcc(), *ARCH, "-shared", *objs, "-o", LIB + ".tmp", "-lcudart"], check=True)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    build(force=True, ptxas_verbose="--ptxas-v" in sys.argv)
    print(LIB)
