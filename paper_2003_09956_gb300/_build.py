"""Compile the CUDA library ``libnsli.so`` in-tree for sm_103a.

nvcc cross-compiles on a machine without a GPU.  The translation units
are compiled in parallel and linked with the static CUDA runtime.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD_DIR = os.path.join(PKG, "_build")
LIB_PATH = os.path.join(BUILD_DIR, "libnsli.so")
SOURCES = ["nsli_kernels.cu", "nsli_api.cu", "nsli_noalloc.cu", "nsli_batch.cu", "nsli_sparse.cu", "nsli_update.cu", "nsli_shard.cu"]
HEADERS = [os.path.join(CSRC, "nsli_internal.h"), os.path.join(CSRC, "nsli_sumsq.cuh"),
           os.path.join(CSRC, "nsli_async.cuh"), os.path.join(INCLUDE, "nsli.h")]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA library cannot be built")


def _stale(target: str, deps: list[str]) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    """Build (if out of date) and return the path of libnsli.so."""
    os.makedirs(BUILD_DIR, exist_ok=True)
    nvcc = _nvcc()
    srcs = [os.path.join(CSRC, s) for s in SOURCES]
    objs = [os.path.join(BUILD_DIR, os.path.splitext(s)[0] + ".o") for s in SOURCES]
    flags = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                    "-I", INCLUDE, "-I", CSRC]
    if verbose:
        flags += ["-Xptxas", "-v"]

    def compile_one(i):
        if force or _stale(objs[i], [srcs[i]] + HEADERS):
            tmp = objs[i] + ".%d.tmp" % os.getpid()
            subprocess.run([nvcc] + flags + ["-c", srcs[i], "-o", tmp], check=True)
            os.replace(tmp, objs[i])

    with cf.ThreadPoolExecutor(len(srcs)) as ex:
        list(ex.map(compile_one, range(len(srcs))))
    if force or _stale(LIB_PATH, objs):
        tmp = LIB_PATH + ".%d.tmp" % os.getpid()
        subprocess.run([nvcc] + ARCH + ["-shared", "-o", tmp] + objs, check=True)
        os.replace(tmp, LIB_PATH)
    return LIB_PATH


if __name__ == "__main__":
    print(build(verbose=True))
