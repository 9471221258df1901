"""Build libhough.so (the CUDA path) in-tree with nvcc for sm_103a.

The library is two translation units -- the C ABI with the kernels
(hough_api.cu) and the host-only request loop (hough_server.cpp) -- linked
against the static CUDA runtime so that the shared object only needs the
driver.
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
DEPS = [SRC, SERVER_SRC, os.path.join(PKG, "csrc", "hough_kernels.cuh"),
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
    os.makedirs(OUT_DIR, exist_ok=True)
    tmp = LIB + f".{os.getpid()}.tmp"
    cmd = [nvcc(), ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-pthread",
           "-shared", "-I", os.path.join(ROOT, "include"), "-o", tmp, SRC, SERVER_SRC, *extra]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        sys.stderr.write(res.stdout + res.stderr)
        raise RuntimeError("nvcc failed building libhough")
    if verbose:
        sys.stderr.write(res.stdout + res.stderr)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(force=True, verbose="-v" in sys.argv)
    print(LIB)
