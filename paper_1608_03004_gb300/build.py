"""Build the CUDA library librlb.so in-tree for sm_103a (GB300) with nvcc.

    python -m paper_1608_03004_gb300.build          # build if a source is newer than the library
    python -m paper_1608_03004_gb300.build --force  # rebuild
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
LIB = os.path.join(PKG, "librlb.so")
SOURCES = [os.path.join(CSRC, "rlb.cu"), os.path.join(CSRC, "rlb_quadrature.cpp")]
DEPS = SOURCES + [os.path.join(CSRC, f) for f in ("rlb_internal.h", "rlb_device_math.cuh", "rlb_stage.cuh",
                                                  "rlb_stage_rp.cuh", "rlb_adjoint.cuh")] + [os.path.join(ROOT, "include", "rlb.h")]
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA library cannot be built")


def cuda_libdir(nv: str) -> str:
    return os.path.join(os.path.dirname(os.path.dirname(os.path.realpath(nv))), "lib64")


def stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(p) > t for p in DEPS)


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile librlb.so next to this file (no-op when it is up to date). Returns its path."""
    if not force and not stale():
        return LIB
    nv = nvcc()
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [nv, ARCH, "-O3", "-lineinfo", "-std=c++17", "-shared", "-Xcompiler", "-fPIC", "--cudart=shared",
           f"-Xlinker=-rpath,{cuda_libdir(nv)}", "-I", os.path.join(ROOT, "include"), "-o", tmp] + SOURCES
    if verbose:
        cmd.insert(2, "-Xptxas=-v")
        print(" ".join(cmd), flush=True)
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
