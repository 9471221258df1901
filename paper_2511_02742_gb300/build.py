"""Build libhough.so (the CUDA path) in-tree with nvcc for sm_103a.

The library is four translation units, compiled in parallel: the C ABI with
the other kernels (hough_api.cu), the fixed-point find kernels
(hough_find.cu), the FP64 variant's find kernel (hough_find_fp64.cu) and the
host-only request loop (hough_server.cpp); they are linked against the static
CUDA runtime so that the shared object only needs the driver.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
SRC = os.path.join(PKG, "csrc", "hough_api.cu")
SERVER_SRC = os.path.join(PKG, "csrc", "hough_server.cpp")
FIND_SRCS = [os.path.join(PKG, "csrc", "hough_find.cu"), os.path.join(PKG, "csrc", "hough_find_fp64.cu")]
UNITS = [SRC, *FIND_SRCS, SERVER_SRC]
DEPS = [*UNITS, os.path.join(PKG, "csrc", "hough_kernels.cuh"),
        os.path.join(PKG, "csrc", "hough_encode.cuh"),
        os.path.join(PKG, "csrc", "hough_internal.h"), os.path.join(PKG, "csrc", "hough_coarse_fine.cuh"),
        os.path.join(PKG, "csrc", "hough_iterative.cuh"),
        os.path.join(PKG, "csrc", "hough_extend.cuh"),
        os.path.join(PKG, "csrc", "hough_slice.cuh"),
        os.path.join(PKG, "csrc", "hough_accumulate.cuh"),
        os.path.join(ROOT, "include", "hough.h")]
OUT_DIR = os.path.join(PKG, "_build")
LIB = os.path.join(OUT_DIR, "libhough.so")
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libhough")


def needs_build() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(d) > t for d in DEPS)


def build(force: bool = False, verbose: bool = False, extra=()) -> str:
    if not force and not needs_build():
        return LIB
    from concurrent.futures import ThreadPoolExecutor
    os.makedirs(OUT_DIR, exist_ok=True)
    tag = f".{os.getpid()}"
    objs = [os.path.join(OUT_DIR, os.path.basename(u) + tag + ".o") for u in UNITS]
    flags = [ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-pthread",
             "-I", os.path.join(ROOT, "include"), *extra]
    if verbose:
        flags.insert(0, "-Xptxas=-v")

    def compile_unit(k):
        return subprocess.run([nvcc(), *flags, "-c", "-o", objs[k], UNITS[k]],
                              capture_output=True, text=True)

    try:
        with ThreadPoolExecutor(len(UNITS)) as ex:
            results = list(ex.map(compile_unit, range(len(UNITS))))
        for res in results:
            if verbose or res.returncode != 0:
                sys.stderr.write(res.stdout + res.stderr)
        if any(res.returncode != 0 for res in results):
            raise RuntimeError("nvcc failed building libhough")
        tmp = LIB + tag + ".tmp"
        res = subprocess.run([nvcc(), ARCH, "-shared", "-Xcompiler", "-pthread", "-o", tmp, *objs],
                             capture_output=True, text=True)
        if res.returncode != 0:
            sys.stderr.write(res.stdout + res.stderr)
            raise RuntimeError("nvcc failed linking libhough")
        os.replace(tmp, LIB)
    finally:
        for o in objs:
            if os.path.exists(o):
                os.remove(o)
    return LIB


if __name__ == "__main__":
    build(force=True, verbose="-v" in sys.argv)
    print(LIB)
