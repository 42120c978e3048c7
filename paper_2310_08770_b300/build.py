"""Builds libccst.so in-tree with nvcc for sm_103a.

Usage: python -m paper_2310_08770_b300.build [--force]
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
import tempfile

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
LIB = os.path.join(PKG, "libccst.so")
SOURCES = ["ccst.cu", "ccst_rois.cu", "ccst_generic.cu", "ccst_mixed.cu", "ccst_peak.cu"] + [f"ccst_track_h{h}.cu" for h in (8, 16, 32, 64, 128)]
DEPS = SOURCES + ["ccst_kernels.cuh", "ccst_device.cuh", "ccst_dfloat.cuh", "ccst_fft.cuh", "ccst_adjoint.cuh",
        "ccst_generic.cuh", "ccst_mixed.cuh", "ccst_mixfft.cuh", "ccst_tc.cuh"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found; the CUDA toolkit is required to build libccst")
    return cand


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, d) for d in DEPS] + [os.path.join(ROOT, "include", "ccst.h")]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile every translation unit (in parallel) and link libccst.so."""
    if not force and not _stale():
        return LIB
    objdir = tempfile.mkdtemp(prefix="ccst_build_")          # objects are not kept: every build compiles all
    flags = [*ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include")]
    if verbose:
        flags.append("-Xptxas=-v")
    procs, objs = [], []
    for src in SOURCES:
        obj = os.path.join(objdir, src.replace(".cu", ".o"))
        objs.append(obj)
        cmd = [nvcc(), *flags, "-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            print(" ".join(cmd))
        procs.append((src, subprocess.Popen(cmd)))
    try:
        failed = [src for src, p in procs if p.wait() != 0]
        if failed:
            raise RuntimeError(f"nvcc failed for {failed}")
        tmp = LIB + ".tmp"
        subprocess.run([nvcc(), *ARCH, "-shared", "-o", tmp] + objs, check=True)
        os.replace(tmp, LIB)
    finally:
        shutil.rmtree(objdir, ignore_errors=True)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
