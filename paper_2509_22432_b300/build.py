"""Build libflood.so (all CUDA sources under csrc/) for sm_103a with nvcc.

The library is built in-tree next to this file. A rebuild happens when any
source or the public header is newer than the library.
"""
from __future__ import annotations

import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(HERE, "libflood.so")
# The bounds-checked build (-DFLOOD_BOUNDS_CHECK): every data-dependent index of
# the kernels is tested before use and reported as a status instead of read or
# written out of range. Loaded instead of LIB when FLOOD_LIBRARY=checked.
LIB_CHECKED = os.path.join(HERE, "libflood_checked.so")

NVCC_FLAGS = [
    "-gencode", "arch=compute_103a,code=sm_103a",
    "-O3", "-lineinfo", "-std=c++17",
    "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
    "--expt-relaxed-constexpr",
    "-shared",
]


def sources() -> list:
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _inputs() -> list:
    return sources() + sorted(glob.glob(os.path.join(CSRC, "*.cuh"))) + [os.path.join(INCLUDE, "flood.h")]


def needs_build(checked: bool = False) -> bool:
    lib = LIB_CHECKED if checked else LIB
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(p) > t for p in _inputs())


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.isabs(c) and os.path.exists(c) or not os.path.isabs(c)):
            return c
    return "nvcc"


def build(force: bool = False, verbose: bool = False, checked: bool = False) -> str:
    """Compile libflood.so (or, checked=True, libflood_checked.so) if needed; returns its path. Raises on failure."""
    lib = LIB_CHECKED if checked else LIB
    if not force and not needs_build(checked):
        return lib
    tmp = lib + f".tmp{os.getpid()}"
    extra = ["-DFLOOD_BOUNDS_CHECK"] if checked else []
    cmd = [nvcc(), *NVCC_FLAGS, *extra, "-I", INCLUDE, "-o", tmp, *sources(), "-lcudart"]
    if verbose:
        print(" ".join(cmd), file=sys.stderr)
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed:\n" + r.stdout + r.stderr)
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, checked="--checked" in sys.argv))
