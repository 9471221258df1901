"""Shared-memory atomic throughput probe: the roofline denominator of the vote
loop, used by bench.py.  Measurement tooling only -- not part of libhough and
not built by the package's build step; compiled here on first use (nvcc,
sm_103a)."""
from __future__ import annotations

import ctypes
import os
import shutil
import subprocess
import sys

_HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(_HERE, "probe.cu")
LIB = os.path.join(_HERE, "_build", "libhough_probe.so")
OPS = {"atom": 0, "red": 1}

_lib = None


def build(force: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    nvcc = os.environ.get("NVCC") or shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    tmp = LIB + f".{os.getpid()}.tmp"
    res = subprocess.run([nvcc, "-gencode=arch=compute_103a,code=sm_103a", "-O3", "-lineinfo",
                          "-std=c++17", "-Xcompiler", "-fPIC", "-shared", "-o", tmp, SRC],
                         capture_output=True, text=True)
    if res.returncode != 0:
        sys.stderr.write(res.stdout + res.stderr)
        raise RuntimeError("nvcc failed building the probe")
    os.replace(tmp, LIB)
    return LIB


def load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        lib.hough_probe_smem_atomics.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                 ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
        lib.hough_probe_smem_atomics.restype = ctypes.c_int
        _lib = lib
    return _lib


def smem_atomic_gops(op: str = "atom", iters: int = 4096, blocks_per_sm: int = 2,
                     threads: int = 1024) -> float:
    """Best of a few runs, in 10^9 shared atomics per second over the whole GPU.
    op "atom": atom.shared.add.u32 with the old value consumed (the vote loop's
    form); op "red": red.shared.add.u32 (no returned value)."""
    lib = load()
    best = 0.0
    for _ in range(3):
        g = ctypes.c_double(0.0)
        ms = ctypes.c_double(0.0)
        rc = lib.hough_probe_smem_atomics(OPS[op], iters, blocks_per_sm, threads,
                                          ctypes.byref(g), ctypes.byref(ms))
        if rc != 0:
            raise RuntimeError(f"smem atomic probe failed ({rc})")
        best = max(best, g.value)
    return best
