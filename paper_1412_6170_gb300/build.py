"""Build the CUDA library ``libknnq.so`` in-tree for sm_103a (GB300).

Each translation unit compiles in its own nvcc process (in parallel), then the
objects are linked into one shared library next to this file under ``_build/``.
``build_debug()`` builds the same sources with ``-DKNN_DEBUG`` (device bounds
checks that record a failure instead of trapping) under ``_build_debug/``; the
binding loads it when the environment variable KNNQ_DEBUG is 1.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libknnq.so")
DEBUG_DIR = os.path.join(HERE, "_build_debug")
DEBUG_LIB = os.path.join(DEBUG_DIR, "libknnq.so")
SOURCES = ["knn_index.cu", "knn_expand.cu", "knn_expand_gather.cu", "knn_expand_tile.cu",
           "knn_expand_wide.cu",
           "knn_expand_iter.cu",
           "knn_brute.cu", "knn_capi.cu", "knn_static.cu", "knn_batch.cu", "knn_server.cu"]
HEADERS = ["knn_device.cuh", "knn_internal.h"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
              "--expt-relaxed-constexpr", "-I", os.path.join(ROOT, "include"), "-I", CSRC]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _deps():
    return ([os.path.join(CSRC, s) for s in SOURCES + HEADERS]
            + [os.path.join(ROOT, "include", "knn.h"), os.path.abspath(__file__)])


def up_to_date(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(d) <= t for d in _deps())


def build(force: bool = False, verbose: bool = False, extra=(), out_dir: str = OUT_DIR) -> str:
    lib = os.path.join(out_dir, "libknnq.so")
    if not force and up_to_date(lib):
        return lib
    os.makedirs(out_dir, exist_ok=True)
    cc = nvcc()

    def compile_one(src):
        obj = os.path.join(out_dir, src.replace(".cu", ".o"))
        cmd = [cc, *ARCH, *NVCC_FLAGS, *extra, "-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            print(" ".join(cmd), flush=True)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        return obj, r.stderr

    with cf.ThreadPoolExecutor(len(SOURCES)) as ex:
        results = list(ex.map(compile_one, SOURCES))
    for _, err in results:
        if verbose and err.strip():
            print(err, flush=True)
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [cc, *ARCH, "-shared", "-cudart", "shared", "-o", tmp, *[o for o, _ in results]]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


def build_debug(force: bool = False, verbose: bool = False) -> str:
    """The library with device bounds checks (-DKNN_DEBUG) under _build_debug/."""
    return build(force=force, verbose=verbose, extra=["-DKNN_DEBUG"], out_dir=DEBUG_DIR)


if __name__ == "__main__":
    v = "-v" in sys.argv
    extra = ["-Xptxas", "-v"] if "--ptxas" in sys.argv else []
    print(build(force=True, verbose=v or bool(extra), extra=extra))
