"""Build the in-tree CUDA library ``libgrace.so`` for sm_103a (GB300).

Each translation unit is compiled by nvcc in parallel, then linked as a shared
library next to this file.  Objects go to ``_build/`` beside the package (ignored
by git).  A rebuild happens only when a source or header is newer than the library.
``build(debug=True)`` makes the checked variant ``libgrace_debug.so`` (-DGRACE_DEBUG:
device-side index checks and workspace guard regions; loaded when GRACE_DEBUG=1).
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
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libgrace.so")
LIB_DEBUG = os.path.join(HERE, "libgrace_debug.so")
SOURCES = ["fastx_q1024.cu", "fastx_q512.cu", "fastx_q128.cu", "fastx_q8.cu", "fastx_q32.cu", "fastyz.cu",
           "fastsplit.cu", "api.cu", "hotpath.cu", "tensor.cu", "fastx.cu", "noalloc.cu", "persist.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I" + INCLUDE]


def nvcc() -> str:
    path = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(path):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libgrace.so")
    return path


def _inputs():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(INCLUDE, "grace.h"))
    return files


def up_to_date(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(f) <= t for f in _inputs())


def build(force: bool = False, verbose: bool = False, debug: bool = False) -> str:
    """Compile and link libgrace.so (debug: libgrace_debug.so); returns its path."""
    lib = LIB_DEBUG if debug else LIB
    if not force and up_to_date(lib):
        return lib
    out = os.path.join(BUILD, "debug") if debug else BUILD
    os.makedirs(out, exist_ok=True)
    cc = nvcc()
    flags = FLAGS + (["-DGRACE_DEBUG"] if debug else [])

    def compile_one(src):
        obj = os.path.join(out, os.path.splitext(src)[0] + ".o")
        cmd = [cc, *ARCH, *flags, "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        if verbose:
            sys.stderr.write(r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = lib + ".tmp"
    r = subprocess.run([cc, *ARCH, "-shared", "-cudart", "static", "-o", tmp, *objs],
                       capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, debug="--debug" in sys.argv))
