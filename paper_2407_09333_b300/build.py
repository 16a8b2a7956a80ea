"""Build ``libhashbatch.so`` in-tree with nvcc for sm_103a (B300).

The library is the whole compute path: the CUDA kernels and the C-ABI of
``include/hashbatch.h``.  Built with ``-gencode arch=compute_103a,code=sm_103a``
only, ``-lineinfo`` for profiler source correlation, and the shared CUDA
runtime so that streams and device pointers are those of the host process.
"""
from __future__ import annotations

import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(PKG, "libhashbatch.so")
SOURCES = ["hb_kernels.cu", "hb_capi.cu", "hb_noalloc.cu", "hb_stream.cu"]
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _deps():
    out = [os.path.join(INCLUDE, "hashbatch.h"), os.path.abspath(__file__)]
    for f in os.listdir(CSRC):
        if f.endswith((".cu", ".cuh", ".h")):
            out.append(os.path.join(CSRC, f))
    return out


def build(force: bool = False, verbose: bool = False, extra=(), out: str | None = None) -> str:
    lib = out or LIB
    if not force and os.path.exists(lib):
        t = os.path.getmtime(lib)
        if all(os.path.getmtime(d) <= t for d in _deps()):
            return lib
    tmp = lib + ".tmp.%d" % os.getpid()
    cmd = [NVCC, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-shared",
           "-Xcompiler", "-fPIC", "-cudart", "shared",
           "-I", INCLUDE, "-I", CSRC, "-o", tmp]
    if verbose:
        cmd += ["-Xptxas", "-v"]
    cmd += list(extra)
    cmd += [os.path.join(CSRC, s) for s in SOURCES]
    subprocess.run(cmd, check=True)
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
