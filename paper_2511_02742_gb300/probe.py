"""Shared-memory atomic throughput probe (the vote loop's ceiling)."""
from __future__ import annotations

import ctypes

from . import build as _build

_lib = None


def load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(_build.build_probe())
        lib.hough_probe_smem_atomics.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                 ctypes.c_void_p, ctypes.c_void_p]
        lib.hough_probe_smem_atomics.restype = ctypes.c_int
        _lib = lib
    return _lib


def smem_atomic_gops(iters: int = 4096, blocks_per_sm: int = 2, threads: int = 1024) -> float:
    """Best of a few runs, in 10^9 shared atomics per second over the whole GPU."""
    lib = load()
    best = 0.0
    for _ in range(3):
        g = ctypes.c_double(0.0)
        ms = ctypes.c_double(0.0)
        rc = lib.hough_probe_smem_atomics(iters, blocks_per_sm, threads, ctypes.byref(g),
                                          ctypes.byref(ms))
        if rc != 0:
            raise RuntimeError(f"smem atomic probe failed ({rc})")
        best = max(best, g.value)
    return best
