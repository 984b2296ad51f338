"""Builds the CUDA library ``libhydro.so`` in-tree for sm_103a (B300).

    python -m paper_1511_02137_b300.build [--verbose] [--checked]

nvcc compiles the kernels and the C ABI into one shared library next to this
file.  Host code is compiled without floating-point contraction so that the
jet positions and cells are the exact FP64 expressions documented in
include/hydro.h.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(HERE, "libhydro.so")
LIB_CHECKED = os.path.join(HERE, "libhydro_check.so")   # -DHYDRO_CHECK: bounds-checked sweeps
SOURCES = ["hydro_api.cu", "hydro_sweep.cu", "hydro_noalloc.cu", "hydro_batch.cu", "hydro_adjoint.cu",
           "hydro_mathcheck.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def _inputs():
    files = [os.path.join(CSRC, s) for s in SOURCES]
    files += [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    files.append(os.path.join(INCLUDE, "hydro.h"))
    return files


def up_to_date(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(f) <= t for f in _inputs())


def build(force: bool = False, verbose: bool = False, checked: bool = False) -> str:
    """Builds libhydro.so, or with `checked` the bounds-checked libhydro_check.so
    (-DHYDRO_CHECK: the sweep tiles check every global cell offset and TMA
    coordinate and report a failure as HYDRO_ECHECK; for tests, not for timing)."""
    lib = LIB_CHECKED if checked else LIB
    if not force and up_to_date(lib):
        return lib
    tmp = lib + ".tmp%d" % os.getpid()
    cmd = [nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-shared", "-Xcompiler", "-fPIC,-ffp-contract=off",
           "-I", INCLUDE, "-I", CSRC, "-o", tmp]
    if checked:
        cmd.append("-DHYDRO_CHECK")
    if verbose:
        cmd += ["-Xptxas", "-v"]
    cmd += [os.path.join(CSRC, s) for s in SOURCES]
    subprocess.check_call(cmd)
    os.replace(tmp, lib)
    return lib


def build_checked(force: bool = False) -> str:
    return build(force=force, checked=True)


if __name__ == "__main__":
    print(build(force=True, verbose="--verbose" in sys.argv, checked="--checked" in sys.argv))
