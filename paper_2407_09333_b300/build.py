"""Build ``libhashbatch.so`` in-tree with nvcc for sm_103a (B300).

The library is the whole compute path: the CUDA kernels and the C-ABI of
``include/hashbatch.h``.  Built with ``-gencode arch=compute_103a,code=sm_103a``
only, ``-lineinfo`` for profiler source correlation, and the shared CUDA
runtime so that streams and device pointers are those of the host process.
"""
from __future__ import annotations

import concurrent.futures
import hashlib
import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(PKG, "libhashbatch.so")
OBJ_DIR = os.path.join(PKG, "_build")
# The hashing kernels' instantiation tables (hb_inst_*.cu) are separate
# translation units so that they compile in parallel.
SOURCES = ["hb_kernels.cu", "hb_capi.cu", "hb_noalloc.cu", "hb_stream.cu",
           "hb_inst_md5.cu", "hb_inst_sha1.cu", "hb_inst_sm3.cu", "hb_inst_all.cu",
           "hb_inst_mixed.cu", "hb_inst_mixed_seg.cu", "hb_inst_relay.cu"]
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC"]


def _headers():
    out = [os.path.join(INCLUDE, "hashbatch.h"), os.path.abspath(__file__)]
    for f in os.listdir(CSRC):
        if f.endswith((".cuh", ".h")):
            out.append(os.path.join(CSRC, f))
    return out


def _stale(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, extra=(), out: str | None = None) -> str:
    """Compiles every source to an object (in parallel, only those older than
    their source or a header) and links the shared library."""
    lib = out or LIB
    headers = _headers()
    srcs = [os.path.join(CSRC, s) for s in SOURCES]
    if not force and not extra and not _stale(lib, headers + srcs):
        return lib
    # objects of a variant build (extra flags) go to their own directory
    tag = "" if not extra else "_" + hashlib.sha256(" ".join(extra).encode()).hexdigest()[:8]
    obj_dir = OBJ_DIR + tag
    os.makedirs(obj_dir, exist_ok=True)
    pid = os.getpid()

    def compile_one(src):
        obj = os.path.join(obj_dir, os.path.basename(src)[:-3] + ".o")
        if force or _stale(obj, headers + [src]):
            cmd = [NVCC, *ARCH, *FLAGS, "-I", INCLUDE, "-I", CSRC, "-c", "-o", obj + ".tmp.%d" % pid]
            if verbose:
                cmd += ["-Xptxas", "-v"]
            cmd += list(extra) + [src]
            subprocess.run(cmd, check=True)
            os.replace(obj + ".tmp.%d" % pid, obj)
        return obj

    workers = max(1, min(len(srcs), os.cpu_count() or 1))
    with concurrent.futures.ThreadPoolExecutor(workers) as ex:
        objs = list(ex.map(compile_one, srcs))
    tmp = lib + ".tmp.%d" % pid
    subprocess.run([NVCC, *ARCH, "-shared", "-cudart", "shared", "-o", tmp, *objs], check=True)
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
