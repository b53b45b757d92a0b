"""Build libeikonal.so in-tree with nvcc for sm_103a (B300).

    python -m paper_2106_15869_b300.build          # rebuild if sources changed
    python -m paper_2106_15869_b300.build --force  # always rebuild

The library is a single translation unit (csrc/eik_api.cu including the
kernel headers); the CUDA runtime is linked statically, so the .so needs only
the driver at run time.
"""
from __future__ import annotations

import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libeikonal.so")
# the same sources with the device-side checks of the debug build (-DEIK_DEBUG)
LIB_DEBUG = os.path.join(HERE, "libeikonal_debug.so")
NVCC_FLAGS = [
    "-gencode", "arch=compute_103a,code=sm_103a",
    "-O3", "-lineinfo", "-std=c++17",
    "-Xcompiler", "-fPIC,-O2",
    "-shared",
]


def sources() -> list[str]:
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cuh"))
                  + [os.path.join(ROOT, "include", "eikonal.h")])


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.isabs(cand) and os.path.exists(cand) or not os.path.isabs(cand)):
            return cand
    return "nvcc"


def needs_build(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(s) > t for s in sources())


def _compile(lib: str, flags: list[str], verbose: bool) -> subprocess.Popen:
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [nvcc(), *NVCC_FLAGS, *flags, "-o", tmp, os.path.join(CSRC, "eik_api.cu")]
    if verbose:
        print(" ".join(cmd), file=sys.stderr)
    return subprocess.Popen(cmd), tmp


def build(force: bool = False, verbose: bool = False, extra_flags: list[str] | None = None,
          debug: bool = True) -> str:
    """Compile csrc/eik_api.cu into libeikonal.so next to this file, and (debug=True) the
    checked build libeikonal_debug.so beside it; the two nvcc runs go in parallel."""
    jobs = []
    if force or needs_build(LIB):
        jobs.append((LIB, *_compile(LIB, list(extra_flags or []), verbose)))
    if debug and (force or needs_build(LIB_DEBUG)):
        jobs.append((LIB_DEBUG, *_compile(LIB_DEBUG, ["-DEIK_DEBUG", *(extra_flags or [])], verbose)))
    for lib, proc, tmp in jobs:
        if proc.wait() != 0:
            raise subprocess.CalledProcessError(proc.returncode, "nvcc " + os.path.basename(lib))
        os.replace(tmp, lib)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True)
    print(LIB)
    print(LIB_DEBUG)
