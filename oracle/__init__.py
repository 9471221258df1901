"""CPU oracle for the track-finding path -- TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package.  The product path (the CUDA library and its
Python binding) never calls it and never falls back to it.

This is a ctypes binding over ``hough_oracle.c`` (plain single-threaded C, see
the header comment there for what it computes and which passage of the paper
each step follows).  The shared object is compiled with gcc on first use.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hough_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

PEAK_DTYPE = np.dtype([("theta", "<u2"), ("rho", "<u2"), ("votes", "<i4"),
                       ("n_hits", "<i4"), ("hit_begin", "<i4")])

CF_DTYPE = np.dtype([(k, "<i4") for k in ("coarse_theta", "coarse_rho", "coarse_votes",
                                            "fine_theta", "fine_rho", "fine_votes", "n_seeds",
                                            "found")])

ITER_DTYPE = np.dtype([(k, "<i4") for k in ("theta", "rho", "votes", "n_hits")])

EXT_DTYPE = np.dtype([(k, "<i4") for k in ("first_vane", "n_hits", "hit_begin", "seed_mid")])

FLAG_FP64 = 2
WIN_PEAK_OVERFLOW = 1
WIN_HIT_OUT_OF_RANGE = 2
WIN_VOTE_OUT_OF_RANGE = 4


class Geometry(ctypes.Structure):
    _fields_ = [("n_vanes", ctypes.c_int32), ("n_z_strips", ctypes.c_int32),
                ("z_pitch_u", ctypes.c_int32), ("z_min_u", ctypes.c_int32),
                ("phi_u_per_deg", ctypes.c_int32), ("z_u_per_mm", ctypes.c_int32),
                ("rho_min", ctypes.c_double), ("rho_max", ctypes.c_double)]


class Thresholds(ctypes.Structure):
    _fields_ = [("vote_threshold", ctypes.c_int32), ("assoc_tol_bins", ctypes.c_int32),
                ("max_peaks", ctypes.c_int32), ("flags", ctypes.c_uint32)]


def build(force: bool = False) -> str:
    """Compile hough_oracle.c into a shared object (gcc, -O2, no -march)."""
    with _lock:
        if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
            os.makedirs(_BUILD, exist_ok=True)
            tmp = _SO + f".{os.getpid()}.tmp"
            subprocess.run(["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-fPIC", "-shared",
                            "-o", tmp, _SRC, "-lm"], check=True)
            os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        i64 = ctypes.c_int64
        i32 = ctypes.c_int
        lib.oracle_tables.argtypes = [P, i32, i32, P, P, P]
        lib.oracle_tables.restype = i32
        lib.oracle_encode.argtypes = [P, P, P, i64, P, P]
        lib.oracle_encode.restype = None
        lib.oracle_vote.argtypes = [P, i32, i32, P, P, i64, P]
        lib.oracle_vote.restype = i64
        lib.oracle_bins_fp64.argtypes = [P, i32, i32, P, P, i64, P]
        lib.oracle_bins_fp64.restype = None
        lib.oracle_bins_fixed.argtypes = [P, i32, i32, P, P, i64, P]
        lib.oracle_bins_fixed.restype = None
        lib.oracle_peaks.argtypes = [P, i32, i32, ctypes.c_int32, ctypes.c_int32, P, P]
        lib.oracle_peaks.restype = ctypes.c_int32
        lib.oracle_find_window.argtypes = [P, i32, i32, P, P, P, i64, P, P, P, P, P, P, P, P]
        lib.oracle_find_window.restype = i32
        lib.oracle_find_batch.argtypes = [P, i32, i32, P, P, P, P, i64, P, P, P, P, P, P, P]
        lib.oracle_find_batch.restype = i32
        lib.oracle_time_slice.argtypes = [P, i64, i64, i64, i64, i64, P, P, i64]
        lib.oracle_time_slice.restype = i64
        lib.oracle_coarse_fine_window.argtypes = [P, P, P, P, i64, P, P]
        lib.oracle_coarse_fine_window.restype = i32
        lib.oracle_coarse_fine_batch.argtypes = [P, P, P, P, P, i64, P, P]
        lib.oracle_coarse_fine_batch.restype = i32
        lib.oracle_iterative_batch.argtypes = [P, i32, i32, P, P, P, P, i64, i32, P, P, P]
        lib.oracle_iterative_batch.restype = i32
        lib.oracle_extend_window.argtypes = [P, P, P, i64, P, ctypes.c_int32, P, P,
                                             ctypes.c_int32, P, P, P]
        lib.oracle_extend_window.restype = i32
        lib.oracle_extend_batch.argtypes = [P, P, P, P, i64, P, P, ctypes.c_int32, P, P,
                                            ctypes.c_int32, P, P, P]
        lib.oracle_extend_batch.restype = i32
        _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def make_geometry(d: dict) -> Geometry:
    return Geometry(d["n_vanes"], d["n_z_strips"], d["z_pitch_u"], d["z_min_u"],
                    d["phi_u_per_deg"], d["z_u_per_mm"], float(d["rho_min"]), float(d["rho_max"]))


def make_thresholds(vote_threshold=5, assoc_tol_bins=1, max_peaks=64, flags=0) -> Thresholds:
    return Thresholds(vote_threshold, assoc_tol_bins, max_peaks, flags)


def tables(geom: dict, n_theta: int, n_rho: int):
    """(C int32[n_theta], S int32[n_theta], D int, K int): fixed-point tables
    at scale 2^K (K the largest <= 24 keeping every box hit's sum in int32)."""
    lib = _load()
    g = make_geometry(geom)
    C = np.zeros(n_theta, np.int32)
    S = np.zeros(n_theta, np.int32)
    D = np.zeros(1, np.int64)
    k = lib.oracle_tables(ctypes.byref(g), n_theta, n_rho, _ptr(C), _ptr(S), _ptr(D))
    if k < 0:
        raise ValueError("bad geometry or shape")
    return C, S, int(D[0]), int(k)


def encode(geom: dict, vane, strip):
    lib = _load()
    g = make_geometry(geom)
    vane = np.ascontiguousarray(vane, np.int32)
    strip = np.ascontiguousarray(strip, np.int32)
    phi = np.zeros(len(vane), np.int32)
    z = np.zeros(len(vane), np.int32)
    lib.oracle_encode(ctypes.byref(g), _ptr(vane), _ptr(strip), len(vane), _ptr(phi), _ptr(z))
    return phi, z


def vote(geom: dict, n_theta: int, n_rho: int, phi_q, z_q):
    """(acc int32[n_theta, n_rho], n_dropped)."""
    lib = _load()
    g = make_geometry(geom)
    phi_q = np.ascontiguousarray(phi_q, np.int32)
    z_q = np.ascontiguousarray(z_q, np.int32)
    acc = np.zeros((n_theta, n_rho), np.int32)
    dropped = lib.oracle_vote(ctypes.byref(g), n_theta, n_rho, _ptr(phi_q), _ptr(z_q),
                              len(phi_q), _ptr(acc))
    return acc, int(dropped)


def bins_fixed(geom: dict, n_theta: int, n_rho: int, phi_q, z_q):
    lib = _load()
    g = make_geometry(geom)
    phi_q = np.ascontiguousarray(phi_q, np.int32)
    z_q = np.ascontiguousarray(z_q, np.int32)
    out = np.zeros((len(phi_q), n_theta), np.int64)
    lib.oracle_bins_fixed(ctypes.byref(g), n_theta, n_rho, _ptr(phi_q), _ptr(z_q), len(phi_q),
                          _ptr(out))
    return out


def bins_fp64(geom: dict, n_theta: int, n_rho: int, phi_q, z_q):
    lib = _load()
    g = make_geometry(geom)
    phi_q = np.ascontiguousarray(phi_q, np.int32)
    z_q = np.ascontiguousarray(z_q, np.int32)
    out = np.zeros((len(phi_q), n_theta), np.int64)
    lib.oracle_bins_fp64(ctypes.byref(g), n_theta, n_rho, _ptr(phi_q), _ptr(z_q), len(phi_q),
                         _ptr(out))
    return out


def peaks(acc, threshold: int, max_peaks: int):
    """Peaks of a given accumulator: (peaks[n_kept] structured, n_found)."""
    lib = _load()
    acc = np.ascontiguousarray(acc, np.int32)
    n_theta, n_rho = acc.shape
    out = np.zeros(max(max_peaks, 1), PEAK_DTYPE)
    kept = np.zeros(1, np.int32)
    found = lib.oracle_peaks(_ptr(acc), n_theta, n_rho, threshold, max_peaks, _ptr(out),
                             _ptr(kept))
    return out[: int(kept[0])].copy(), int(found)


def find_window(geom: dict, n_theta: int, n_rho: int, phi_q, z_q, vote_threshold=5,
                assoc_tol_bins=1, max_peaks=64, fp64=False):
    """One window through voting, peaks and association; returns a dict.
    fp64: bins from Eq. (1) in double precision instead of the tables."""
    lib = _load()
    g = make_geometry(geom)
    th = make_thresholds(vote_threshold, assoc_tol_bins, max_peaks, FLAG_FP64 if fp64 else 0)
    phi_q = np.ascontiguousarray(phi_q, np.int32)
    z_q = np.ascontiguousarray(z_q, np.int32)
    n = len(phi_q)
    acc = np.zeros((n_theta, n_rho), np.int32)
    dropped = np.zeros(1, np.int64)
    pk = np.zeros(max(max_peaks, 1), PEAK_DTYPE)
    n_peaks = np.zeros(1, np.int32)
    n_found = np.zeros(1, np.int32)
    hit_track = np.zeros(n, np.int32)
    track_hits = np.zeros(n, np.int32)
    status = np.zeros(1, np.uint32)
    rc = lib.oracle_find_window(ctypes.byref(g), n_theta, n_rho, ctypes.byref(th), _ptr(phi_q),
                                _ptr(z_q), n, _ptr(acc), _ptr(dropped), _ptr(pk), _ptr(n_peaks),
                                _ptr(n_found), _ptr(hit_track), _ptr(track_hits), _ptr(status))
    if rc != 0:
        raise ValueError("oracle_find_window: bad arguments")
    k = int(n_peaks[0])
    return dict(acc=acc, n_dropped=int(dropped[0]), peaks=pk[:k].copy(), n_peaks=k,
                n_found=int(n_found[0]), hit_track=hit_track, track_hits=track_hits,
                status=int(status[0]))


def find_batch(geom: dict, n_theta: int, n_rho: int, phi_q, z_q, offsets, vote_threshold=5,
               assoc_tol_bins=1, max_peaks=64, export_acc=False, fp64=False):
    """A CSR batch of windows; outputs in the library's layout (dict of arrays).
    fp64: bins from Eq. (1) in double precision instead of the tables."""
    lib = _load()
    g = make_geometry(geom)
    th = make_thresholds(vote_threshold, assoc_tol_bins, max_peaks, FLAG_FP64 if fp64 else 0)
    phi_q = np.ascontiguousarray(phi_q, np.int32)
    z_q = np.ascontiguousarray(z_q, np.int32)
    offsets = np.ascontiguousarray(offsets, np.int64)
    nw = len(offsets) - 1
    n = len(phi_q)
    acc = np.zeros((nw, n_theta, n_rho), np.int32) if export_acc else None
    pk = np.zeros(nw * max(max_peaks, 0), PEAK_DTYPE)
    n_peaks = np.zeros(nw, np.int32)
    n_found = np.zeros(nw, np.int32)
    hit_track = np.zeros(n, np.int32)
    track_hits = np.zeros(n, np.int32)
    status = np.zeros(nw, np.uint32)
    rc = lib.oracle_find_batch(ctypes.byref(g), n_theta, n_rho, ctypes.byref(th), _ptr(phi_q),
                               _ptr(z_q), _ptr(offsets), nw, _ptr(acc), _ptr(pk), _ptr(n_peaks),
                               _ptr(n_found), _ptr(hit_track), _ptr(track_hits), _ptr(status))
    if rc != 0:
        raise ValueError("oracle_find_batch: bad arguments")
    return dict(acc=acc, peaks=pk.reshape(nw, max_peaks) if max_peaks else pk.reshape(nw, 0),
                n_peaks=n_peaks, n_found=n_found, hit_track=hit_track, track_hits=track_hits,
                status=status)


def time_slice(t, t0: int, step: int, length: int, n_windows: int):
    """Overlapping time windows (Section 5): (offsets int64[n_windows+1],
    index int64[m]) -- window k holds the input positions of the hits with
    t0 + k*step <= t < t0 + k*step + length, in input order."""
    lib = _load()
    t = np.ascontiguousarray(t, np.int64)
    offsets = np.zeros(n_windows + 1, np.int64)
    cap = max(1, len(t) * (-(-length // step)))
    index = np.zeros(cap, np.int64)
    m = lib.oracle_time_slice(_ptr(t), len(t), t0, step, length, n_windows, _ptr(offsets),
                              _ptr(index), cap)
    if m < 0:
        raise ValueError(f"oracle_time_slice: error {m}")
    return offsets, index[:m].copy()


def coarse_fine(geom: dict, phi_q, z_q, offsets, vote_threshold=5, assoc_tol_bins=1):
    """The paper's coarse (18 x 100) then fine (10 x 10 of the 180 x 1000 grid)
    search, one line per window: (result[n_windows] CF_DTYPE, hit_track)."""
    lib = _load()
    g = make_geometry(geom)
    th = make_thresholds(vote_threshold, assoc_tol_bins, 0)
    phi_q = np.ascontiguousarray(phi_q, np.int32)
    z_q = np.ascontiguousarray(z_q, np.int32)
    offsets = np.ascontiguousarray(offsets, np.int64)
    nw = len(offsets) - 1
    out = np.zeros(nw, CF_DTYPE)
    ht = np.zeros(max(len(phi_q), 1), np.int32)
    rc = lib.oracle_coarse_fine_batch(ctypes.byref(g), ctypes.byref(th), _ptr(phi_q), _ptr(z_q),
                                      _ptr(offsets), nw, _ptr(out), _ptr(ht))
    if rc != 0:
        raise ValueError("oracle_coarse_fine_batch: bad arguments")
    return out, ht[:len(phi_q)]


def iterative(geom: dict, n_theta: int, n_rho: int, phi_q, z_q, offsets, max_tracks=64,
              vote_threshold=5, assoc_tol_bins=1):
    """Highest bin, assign its line's hits, remove them, vote again (the literal
    reading of the paper's peak step): (tracks[n_windows, max_tracks] ITER_DTYPE,
    n_tracks[n_windows], hit_track[n_hits])."""
    lib = _load()
    g = make_geometry(geom)
    th = make_thresholds(vote_threshold, assoc_tol_bins, 0)
    phi_q = np.ascontiguousarray(phi_q, np.int32)
    z_q = np.ascontiguousarray(z_q, np.int32)
    offsets = np.ascontiguousarray(offsets, np.int64)
    nw = len(offsets) - 1
    tracks = np.zeros((nw, max(max_tracks, 1)), ITER_DTYPE)
    n_tracks = np.zeros(nw, np.int32)
    ht = np.zeros(max(len(phi_q), 1), np.int32)
    rc = lib.oracle_iterative_batch(ctypes.byref(g), n_theta, n_rho, ctypes.byref(th), _ptr(phi_q),
                                    _ptr(z_q), _ptr(offsets), nw, max_tracks, _ptr(tracks),
                                    _ptr(n_tracks), _ptr(ht))
    if rc != 0:
        raise ValueError("oracle_iterative_batch: bad arguments")
    return tracks, n_tracks, ht[:len(phi_q)]


def extend(geom: dict, phi_q, z_q, offsets, found: dict, tol_z: int):
    """Track extension (Section 4) of a CSR batch, from the output of
    find_batch on the same hits: (ext[n_windows, max_peaks] EXT_DTYPE,
    ext_track[n_hits], ext_hits[n_hits]), per-hit arrays window-local."""
    lib = _load()
    g = make_geometry(geom)
    phi_q = np.ascontiguousarray(phi_q, np.int32)
    z_q = np.ascontiguousarray(z_q, np.int32)
    offsets = np.ascontiguousarray(offsets, np.int64)
    nw = len(offsets) - 1
    pk = np.ascontiguousarray(found["peaks"])
    max_peaks = pk.shape[1]
    n_peaks = np.ascontiguousarray(found["n_peaks"], np.int32)
    hit_track = np.ascontiguousarray(found["hit_track"], np.int32)
    track_hits = np.ascontiguousarray(found["track_hits"], np.int32)
    ext = np.zeros((nw, max(max_peaks, 1)), EXT_DTYPE)
    n = len(phi_q)
    ext_track = np.zeros(max(n, 1), np.int32)
    ext_hits = np.zeros(max(n, 1), np.int32)
    rc = lib.oracle_extend_batch(ctypes.byref(g), _ptr(phi_q), _ptr(z_q), _ptr(offsets), nw,
                                 _ptr(pk), _ptr(n_peaks), max_peaks, _ptr(hit_track),
                                 _ptr(track_hits), int(tol_z), _ptr(ext), _ptr(ext_track),
                                 _ptr(ext_hits))
    if rc != 0:
        raise ValueError("oracle_extend_batch: bad arguments")
    return ext[:, :max_peaks], ext_track[:n], ext_hits[:n]


def extend_window(geom: dict, phi_q, z_q, groups, tol_z: int, rejected=()):
    """Track extension of one window from given step-D groups: `groups` is a
    list (in peak order) of lists of hit indices in increasing order; hits in
    `rejected` are marked as rejected by the find step.  Returns
    (ext[len(groups)] EXT_DTYPE, ext_track, ext_hits)."""
    lib = _load()
    g = make_geometry(geom)
    phi_q = np.ascontiguousarray(phi_q, np.int32)
    z_q = np.ascontiguousarray(z_q, np.int32)
    n = len(phi_q)
    pk = np.zeros(max(len(groups), 1), PEAK_DTYPE)
    hit_track = np.full(max(n, 1), -1, np.int32)
    hit_track[list(rejected)] = -2
    assert not set(rejected) & {h for g_ in groups for h in g_}, "rejected hits have no group"
    order = []
    assert sum(len(g_) for g_ in groups) == len({h for g_ in groups for h in g_}), \
        "step-D groups are disjoint"
    for p, grp in enumerate(groups):
        pk[p]["hit_begin"] = len(order)
        pk[p]["n_hits"] = len(grp)
        order += list(grp)
        hit_track[list(grp)] = p
    order += [h for h in range(n) if h not in set(order)]
    track_hits = np.zeros(max(n, 1), np.int32)
    track_hits[:n] = order
    ext = np.zeros(max(len(groups), 1), EXT_DTYPE)
    ext_track = np.zeros(max(n, 1), np.int32)
    ext_hits = np.zeros(max(n, 1), np.int32)
    rc = lib.oracle_extend_window(ctypes.byref(g), _ptr(phi_q), _ptr(z_q), n, _ptr(pk),
                                  len(groups), _ptr(hit_track), _ptr(track_hits), int(tol_z),
                                  _ptr(ext), _ptr(ext_track), _ptr(ext_hits))
    if rc != 0:
        raise ValueError("oracle_extend_window: bad arguments")
    return ext[:len(groups)], ext_track[:n], ext_hits[:n]
