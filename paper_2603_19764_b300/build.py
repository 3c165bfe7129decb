"""Build libsph.so in-tree with nvcc for sm_103a (B300).

    python -m paper_2603_19764_b300.build [--force] [--verbose] [--checked]
"""
from __future__ import annotations

import glob
import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(PKG, "libsph.so")
# the checked build: index tests on every data-derived index (-DSPH_BOUNDS_CHECK)
LIB_CHECKED = os.path.join(PKG, "libsph_check.so")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _inputs():
    return sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(INCLUDE, "*.h"))


def is_stale(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(f) > t for f in _inputs())


def command(out: str = LIB, verbose: bool = False, checked: bool = False):
    cmd = [NVCC, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2",
           "-shared", "-I", INCLUDE, "-o", out, *sources()]
    if checked:
        cmd.insert(1, "-DSPH_BOUNDS_CHECK")
    if verbose:
        cmd += ["-Xptxas", "-v"]
    return cmd


def build(force: bool = False, verbose: bool = False, checked: bool = False) -> str:
    """Build libsph.so (or, checked = True, libsph_check.so: the same
    library with an index test before every access whose index comes from
    data; a failed test is reported as SPH_E_INTERNAL instead of faulting)."""
    lib = LIB_CHECKED if checked else LIB
    if force or is_stale(lib):
        tmp = lib + ".tmp%d" % os.getpid()
        subprocess.check_call(command(tmp, verbose, checked))
        os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="--verbose" in sys.argv,
                checked="--checked" in sys.argv))
