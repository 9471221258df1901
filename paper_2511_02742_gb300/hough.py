"""Python binding of libhough (include/hough.h): argument marshalling only.

Every step of the path runs in the CUDA library; this module only converts
torch tensors / numpy arrays to the C structs and pointers of the C ABI.  If
the library has not been built, loading fails loudly: there is no fallback.

The function names follow the C ABI (hough_create, hough_find, ...); the
``Finder`` class bundles a context with output allocation for torch users.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

HOUGH_OK = 0
HOUGH_MAX_FRAC_BITS = 24
HOUGH_MAX_THETA = 4096
HOUGH_MAX_RHO = 1024
HOUGH_MAX_PEAKS = 256
HOUGH_NOALLOC_MAX_THETA = 4096
HOUGH_WIN_PEAK_OVERFLOW = 1
HOUGH_WIN_HIT_OUT_OF_RANGE = 2
HOUGH_WIN_VOTE_OUT_OF_RANGE = 4
HOUGH_WIN_BAD_OFFSETS = 8
HOUGH_WIN_TOO_LARGE = 16
HOUGH_ITER_MAX_HITS = 4096
HOUGH_EXT_MAX_HITS = 4096
HOUGH_EXT_MAX_VANES = 256
HOUGH_EXT_MAX_TOL = (1 << 19) - 1
HOUGH_FLAG_EXPORT_ACC = 1
HOUGH_FLAG_FP64 = 2
HOUGH_ERR_INVALID_ARG = -1
HOUGH_ERR_TIMEOUT = -4
HOUGH_ERR_UNSUPPORTED_SHAPE = -5
HOUGH_ERR_BUSY = -7
HOUGH_SLICE_MAX_OVERLAP = 16
HOUGH_SLICE_UNSORTED = 1

PEAK_DTYPE = np.dtype([("theta", "<u2"), ("rho", "<u2"), ("votes", "<i4"),
                       ("n_hits", "<i4"), ("hit_begin", "<i4")])

P = ctypes.c_void_p


class hough_geometry(ctypes.Structure):
    _fields_ = [("n_vanes", ctypes.c_int32), ("n_z_strips", ctypes.c_int32),
                ("z_pitch_u", ctypes.c_int32), ("z_min_u", ctypes.c_int32),
                ("phi_u_per_deg", ctypes.c_int32), ("z_u_per_mm", ctypes.c_int32),
                ("rho_min", ctypes.c_double), ("rho_max", ctypes.c_double)]


class hough_thresholds(ctypes.Structure):
    _fields_ = [("vote_threshold", ctypes.c_int32), ("assoc_tol_bins", ctypes.c_int32),
                ("max_peaks", ctypes.c_int32), ("flags", ctypes.c_uint32)]


class hough_hits(ctypes.Structure):
    _fields_ = [("phi_q", P), ("z_q", P), ("vane", P), ("strip", P), ("n_hits", ctypes.c_int64)]


class hough_tracks(ctypes.Structure):
    _fields_ = [("peaks", P), ("n_peaks", P), ("n_found", P), ("hit_track", P),
                ("track_hits", P), ("window_status", P), ("acc", P)]


class hough_launch(ctypes.Structure):
    _fields_ = [("threads", ctypes.c_int32), ("word_rows", ctypes.c_int32),
                ("hit_stage", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32)]

    def as_dict(self):
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


class hough_server_config(ctypes.Structure):
    _fields_ = [("n_slots", ctypes.c_int32), ("raw_hits", ctypes.c_int32),
                ("slot_windows", ctypes.c_int64), ("slot_hits", ctypes.c_int64),
                ("max_queued", ctypes.c_int64), ("launch", hough_launch)]


class hough_request(ctypes.Structure):
    _fields_ = [("in0", P), ("in1", P), ("window_offsets", P), ("n_windows", ctypes.c_int64),
                ("out", hough_tracks), ("arrival_ns", ctypes.c_int64)]


class hough_request_result(ctypes.Structure):
    _fields_ = [("ticket", ctypes.c_uint64), ("status", ctypes.c_int32),
                ("batch_requests", ctypes.c_int32), ("batch_windows", ctypes.c_int64),
                ("arrival_ns", ctypes.c_int64), ("launch_ns", ctypes.c_int64),
                ("done_ns", ctypes.c_int64), ("pack_ns", ctypes.c_int64),
                ("h2d_ns", ctypes.c_int64), ("kernel_ns", ctypes.c_int64),
                ("d2h_ns", ctypes.c_int64), ("scatter_ns", ctypes.c_int64)]

    def as_dict(self):
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


class hough_server_stats(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int64) for k in ("submitted", "rejected", "completed", "queued",
                                               "in_flight", "batches", "windows",
                                               "device_bytes", "host_bytes")]

    def as_dict(self):
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


class HoughError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: {status_string(code)} ({code})")
        self.code = code


_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Load libhough.so; raise if it is missing (no CPU fallback exists)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_build.LIB):
        if not build_if_missing:
            raise RuntimeError(f"CUDA library not built ({_build.LIB} missing); "
                               "run `python -c 'import __graft_entry__ as g; g.build()'`")
        _build.build()
    lib = ctypes.CDLL(_build.LIB)
    i32, i64 = ctypes.c_int, ctypes.c_int64
    sig = {
        "hough_tables": ([P, i32, i32, P, P, P, P], i32),
        "hough_tile_bins": ([P, i32, i32, i32, P, P], i32),
        "hough_create": ([P, i32, i32, P, P], i32),
        "hough_destroy": ([P], None),
        "hough_encode": ([P, P, P, i64, P, P, P], i32),
        "hough_find": ([P, P, P, i64, P, P], i32),
        "hough_find_host": ([P, P, P, i64, P, P], i32),
        "hough_plan_create": ([P, P, P, i64, P, P, P], i32),
        "hough_plan_launch": ([P, P], i32),
        "hough_plan_destroy": ([P], None),
        "hough_get_launch": ([P, P], i32),
        "hough_set_launch": ([P, P], i32),
        "hough_autotune": ([P, P, P, i64, P, P, i32, P], i32),
        "hough_find_noalloc": ([P, i32, i32, P, P, P, i64, P, P], i32),
        "hough_status_string": ([i32], ctypes.c_char_p),
        "hough_last_error": ([P], i32),
        "hough_launch_count": ([P], i64),
        "hough_find_coarse_fine": ([P, P, P, i64, P, P, P], i32),
        "hough_find_iterative": ([P, P, P, i64, ctypes.c_int32, P, P, P, P, P], i32),
        "hough_accumulate": ([P, P, P, i64, P, P, P], i32),
        "hough_time_slice": ([P, P, P, P, i64, i64, i64, i64, i64, P, P, P, i64, P, P, P], i32),
        "hough_extend": ([P, P, P, i64, P, ctypes.c_int32, P, P], i32),
        "hough_server_create": ([P, P, P], i32),
        "hough_server_submit": ([P, P, P], i32),
        "hough_server_wait": ([P, ctypes.c_uint64, i64, P], i32),
        "hough_server_poll": ([P, P, i64, P], i32),
        "hough_server_drain": ([P, i64], i32),
        "hough_server_get_stats": ([P, P], i32),
        "hough_server_destroy": ([P], None),
        "hough_server_clock_ns": ([], i64),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


def status_string(code: int) -> str:
    try:
        return load().hough_status_string(int(code)).decode()
    except Exception:  # pragma: no cover - library missing
        return "HOUGH_ERR"


def _check(code: int, what: str):
    if code != HOUGH_OK:
        raise HoughError(code, what)


def make_geometry(d: dict) -> hough_geometry:
    return hough_geometry(d["n_vanes"], d["n_z_strips"], d["z_pitch_u"], d["z_min_u"],
                          d["phi_u_per_deg"], d["z_u_per_mm"], float(d["rho_min"]),
                          float(d["rho_max"]))


def _ptr(x):
    """Address of a torch tensor or numpy array (None -> NULL)."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        return ctypes.c_void_p(x.data_ptr())
    return x.ctypes.data_as(ctypes.c_void_p)


def _stream(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


# ----------------------------------------------------------- C-ABI functions

def hough_tables(geometry: dict, n_theta: int, n_rho: int):
    """Host-only fixed-point tables: (C int32[n_theta], S int32[n_theta], D, K)."""
    lib = load()
    g = make_geometry(geometry)
    C = np.zeros(n_theta, np.int32)
    S = np.zeros(n_theta, np.int32)
    D = np.zeros(1, np.int64)
    K = np.zeros(1, np.int32)
    _check(lib.hough_tables(ctypes.byref(g), n_theta, n_rho, _ptr(C), _ptr(S), _ptr(D), _ptr(K)),
           "hough_tables")
    return C, S, int(D[0]), int(K[0])


def hough_tile_bins(geometry: dict, n_theta: int, n_rho: int, word_rows: int):
    """Host-only narrowed-tile layout of the find: (NB, lo int32[3, ceil(n_theta/32)]),
    lo[k, i] the first stored bin of tile i with 2^k counters per word."""
    lib = load()
    g = make_geometry(geometry)
    nb = np.zeros(1, np.int32)
    lo = np.zeros(3 * ((n_theta + 31) // 32), np.int32)
    _check(lib.hough_tile_bins(ctypes.byref(g), n_theta, n_rho, word_rows, _ptr(nb), _ptr(lo)),
           "hough_tile_bins")
    return int(nb[0]), lo.reshape(3, -1)


def hough_create(geometry: dict, n_theta: int, n_rho: int, vote_threshold=5, assoc_tol_bins=1,
                 max_peaks=64, flags=0) -> ctypes.c_void_p:
    lib = load()
    g = make_geometry(geometry)
    th = hough_thresholds(vote_threshold, assoc_tol_bins, max_peaks, flags)
    ctx = ctypes.c_void_p()
    _check(lib.hough_create(ctypes.byref(g), n_theta, n_rho, ctypes.byref(th), ctypes.byref(ctx)),
           "hough_create")
    return ctx


def hough_destroy(ctx) -> None:
    load().hough_destroy(ctx)


def _check_buf(x, dtype, min_numel: int, cuda: bool, name: str) -> None:
    """A buffer handed to the library must be a contiguous torch tensor of the
    given dtype, on the GPU (device entry points) or in host memory (host
    entry points), with at least min_numel elements: the kernels trust the
    pointers and sizes they get."""
    import torch
    if not isinstance(x, torch.Tensor):
        raise TypeError(f"{name}: a torch tensor is needed, got {type(x).__name__}")
    if x.dtype != dtype:
        raise TypeError(f"{name}: dtype {x.dtype}, expected {dtype}")
    if not x.is_contiguous():
        raise ValueError(f"{name}: must be contiguous")
    if x.is_cuda != cuda:
        raise ValueError(f"{name}: must be {'on the GPU' if cuda else 'in host memory'}")
    if x.numel() < min_numel:
        raise ValueError(f"{name}: {x.numel()} elements, at least {min_numel} needed")


def _check_host(x, dtype, min_numel: int, name: str) -> None:
    """A host buffer: a contiguous numpy array, or a torch tensor in host
    memory, of the given dtype and at least min_numel elements."""
    if isinstance(x, np.ndarray):
        ok = x.dtype == dtype and x.flags.c_contiguous
        size = x.size
    elif hasattr(x, "is_cuda") and hasattr(x, "numpy"):
        ok = (not x.is_cuda) and x.is_contiguous() and x.numpy().dtype == dtype
        size = int(x.numel())
    else:
        ok, size = False, 0
    if not ok:
        raise TypeError(f"{name}: a contiguous host array of {np.dtype(dtype)} is needed")
    if size < min_numel:
        raise ValueError(f"{name}: {size} elements, at least {min_numel} needed")


def _check_hits(hits: dict, cuda: bool) -> int:
    import torch
    keys = ("vane", "strip") if "vane" in hits else ("phi_q", "z_q")
    n = int(hits[keys[0]].numel()) if hasattr(hits[keys[0]], "numel") else -1
    for k in keys:
        _check_buf(hits[k], torch.int32, n, cuda, k)
    if int(hits[keys[1]].numel()) != n:
        raise ValueError(f"{keys[0]} and {keys[1]} differ in length")
    return n


def _check_outputs(out: dict, n_windows: int, n_hits: int, max_peaks: int, export: tuple | None,
                   cuda: bool) -> None:
    import torch
    i32 = torch.int32
    if max_peaks > 0:
        _check_buf(out.get("peaks"), i32, n_windows * max_peaks * 4, cuda, "peaks")
    _check_buf(out.get("n_peaks"), i32, n_windows, cuda, "n_peaks")
    if out.get("n_found") is not None:
        _check_buf(out["n_found"], i32, n_windows, cuda, "n_found")
    _check_buf(out.get("window_status"), i32, n_windows, cuda, "window_status")
    _check_buf(out.get("hit_track"), i32, n_hits, cuda, "hit_track")
    _check_buf(out.get("track_hits"), i32, n_hits, cuda, "track_hits")
    if export is not None:
        _check_buf(out.get("acc"), i32, n_windows * export[0] * export[1], cuda, "acc")


def make_hits(phi_q=None, z_q=None, vane=None, strip=None, n_hits=None) -> hough_hits:
    if n_hits is None:
        n_hits = len(vane) if vane is not None else len(phi_q)
    return hough_hits(_ptr(phi_q), _ptr(z_q), _ptr(vane), _ptr(strip), int(n_hits))


def make_tracks(out: dict) -> hough_tracks:
    return hough_tracks(_ptr(out.get("peaks")), _ptr(out["n_peaks"]), _ptr(out.get("n_found")),
                        _ptr(out["hit_track"]), _ptr(out["track_hits"]),
                        _ptr(out["window_status"]), _ptr(out.get("acc")))


def hough_encode(ctx, vane, strip, phi_q, z_q, stream=None) -> None:
    _check(load().hough_encode(ctx, _ptr(vane), _ptr(strip), len(vane), _ptr(phi_q), _ptr(z_q),
                               _stream(stream)), "hough_encode")


LINE_DTYPE = np.dtype([(k, "<i4") for k in ("coarse_theta", "coarse_rho", "coarse_votes",
                                              "fine_theta", "fine_rho", "fine_votes", "n_seeds",
                                              "found")])


def hough_find_coarse_fine(ctx, hits: hough_hits, window_offsets, n_windows: int, lines,
                           hit_track, stream=None) -> None:
    """The paper's coarse (18 x 100) then fine (10 x 10) search, one line per
    window; lines: int32 tensor [n_windows, 8] (hough_line)."""
    _check(load().hough_find_coarse_fine(ctx, ctypes.byref(hits), _ptr(window_offsets), n_windows,
                                         _ptr(lines), _ptr(hit_track), _stream(stream)),
           "hough_find_coarse_fine")


def hough_accumulate(ctx, hits: hough_hits, window_offsets, n_windows: int, acc, window_status,
                     stream=None) -> None:
    """Steps A-B with every window's accumulator written out;
    acc: int32 tensor [n_windows, n_theta, n_rho]."""
    _check(load().hough_accumulate(ctx, ctypes.byref(hits), _ptr(window_offsets), int(n_windows),
                                   _ptr(acc), _ptr(window_status), _stream(stream)),
           "hough_accumulate")


ITER_DTYPE = np.dtype([(k, "<i4") for k in ("theta", "rho", "votes", "n_hits")])


def hough_find_iterative(ctx, hits: hough_hits, window_offsets, n_windows: int, max_tracks: int,
                         tracks, n_tracks, hit_track, window_status, stream=None) -> None:
    """Iterative highest-bin search; tracks: int32 tensor [n_windows, max_tracks, 4]."""
    _check(load().hough_find_iterative(ctx, ctypes.byref(hits), _ptr(window_offsets), n_windows,
                                       max_tracks, _ptr(tracks), _ptr(n_tracks), _ptr(hit_track),
                                       _ptr(window_status), _stream(stream)),
           "hough_find_iterative")


EXT_DTYPE = np.dtype([(k, "<i4") for k in ("first_vane", "n_hits", "hit_begin", "seed_mid")])


class hough_extension(ctypes.Structure):
    _fields_ = [("tracks", P), ("ext_track", P), ("ext_hits", P), ("window_status", P)]


def hough_extend(ctx, hits: hough_hits, window_offsets, n_windows: int, found: hough_tracks,
                 tol_z: int, out: dict, stream=None) -> None:
    """Track extension on hough_find's outputs; out: dict of device tensors
    tracks [n_windows, max_peaks, 4], ext_track, ext_hits, window_status."""
    ext = hough_extension(_ptr(out["tracks"]), _ptr(out["ext_track"]), _ptr(out["ext_hits"]),
                          _ptr(out["window_status"]))
    _check(load().hough_extend(ctx, ctypes.byref(hits), _ptr(window_offsets), int(n_windows),
                               ctypes.byref(found), int(tol_z), ctypes.byref(ext),
                               _stream(stream)), "hough_extend")


def hough_time_slice(ctx, t, in0, in1, t0: int, step: int, length: int, n_windows: int,
                     out0, out1, out_index, window_offsets, status=None, stream=None) -> None:
    """Overlapping time windows on the device (device tensors; see hough.h)."""
    n = int(t.numel())
    cap = int(out0.numel())
    _check(load().hough_time_slice(ctx, _ptr(t), _ptr(in0), _ptr(in1), n, int(t0), int(step),
                                   int(length), int(n_windows), _ptr(out0), _ptr(out1),
                                   _ptr(out_index), cap, _ptr(window_offsets), _ptr(status),
                                   _stream(stream)), "hough_time_slice")


def hough_find(ctx, hits: hough_hits, window_offsets, n_windows: int, tracks_out: hough_tracks,
               stream=None) -> None:
    _check(load().hough_find(ctx, ctypes.byref(hits), _ptr(window_offsets), int(n_windows),
                             ctypes.byref(tracks_out), _stream(stream)), "hough_find")


def hough_find_host(ctx, hits: hough_hits, window_offsets, n_windows: int,
                    tracks_out: hough_tracks, stream=None) -> None:
    _check(load().hough_find_host(ctx, ctypes.byref(hits), _ptr(window_offsets), int(n_windows),
                                  ctypes.byref(tracks_out), _stream(stream)), "hough_find_host")


def hough_plan_create(ctx, hits: hough_hits, window_offsets, n_windows: int,
                      tracks_out: hough_tracks, stream=None) -> ctypes.c_void_p:
    plan = ctypes.c_void_p()
    _check(load().hough_plan_create(ctx, ctypes.byref(hits), _ptr(window_offsets), int(n_windows),
                                    ctypes.byref(tracks_out), _stream(stream), ctypes.byref(plan)),
           "hough_plan_create")
    return plan


def hough_plan_launch(plan, stream=None) -> None:
    _check(load().hough_plan_launch(plan, _stream(stream)), "hough_plan_launch")


def hough_plan_destroy(plan) -> None:
    load().hough_plan_destroy(plan)


def hough_get_launch(ctx) -> dict:
    l = hough_launch()
    _check(load().hough_get_launch(ctx, ctypes.byref(l)), "hough_get_launch")
    return l.as_dict()


def hough_set_launch(ctx, threads=0, word_rows=0, hit_stage=0, ctas_per_sm=0) -> None:
    l = hough_launch(threads, word_rows, hit_stage, ctas_per_sm)
    _check(load().hough_set_launch(ctx, ctypes.byref(l)), "hough_set_launch")


def hough_autotune(ctx, hits: hough_hits, window_offsets, n_windows: int,
                   tracks_out: hough_tracks, iters=3, stream=None) -> dict:
    l = hough_launch()
    _check(load().hough_autotune(ctx, ctypes.byref(hits), _ptr(window_offsets), int(n_windows),
                                 ctypes.byref(tracks_out), _stream(stream), int(iters),
                                 ctypes.byref(l)), "hough_autotune")
    return l.as_dict()


def hough_find_noalloc(geometry: dict, n_theta: int, n_rho: int, hits: hough_hits, window_offsets,
                       n_windows: int, tracks_out: hough_tracks, vote_threshold=5,
                       assoc_tol_bins=1, max_peaks=64, flags=0, stream=None) -> None:
    """hough_find without a context and without any allocation (see the C
    header): tables and counters live in the library's fixed device array."""
    g = make_geometry(geometry)
    th = hough_thresholds(vote_threshold, assoc_tol_bins, max_peaks, flags)
    _check(load().hough_find_noalloc(ctypes.byref(g), n_theta, n_rho, ctypes.byref(th),
                                     ctypes.byref(hits), _ptr(window_offsets), int(n_windows),
                                     ctypes.byref(tracks_out), _stream(stream)),
           "hough_find_noalloc")


def hough_last_error(ctx) -> int:
    return int(load().hough_last_error(ctx))


def hough_launch_count(ctx) -> int:
    return int(load().hough_launch_count(ctx))


# ------------------------------------------------------------ torch helper

def decode_peaks(peaks_i32) -> np.ndarray:
    """int32[..., 4] peak records (as written by the library) -> PEAK_DTYPE array."""
    a = np.ascontiguousarray(peaks_i32.cpu().numpy() if hasattr(peaks_i32, "cpu") else peaks_i32,
                             dtype=np.int32)
    return a.view(PEAK_DTYPE).reshape(a.shape[:-1])


class Finder:
    """One context (accumulator shape + thresholds) on the current CUDA device."""

    def __init__(self, n_theta: int, n_rho: int, geometry: dict | None = None, vote_threshold=5,
                 assoc_tol_bins=1, max_peaks=64, export_acc=False, fp64=False):
        from .synth import GEOMETRY
        self.geometry = dict(GEOMETRY if geometry is None else geometry)
        self.n_theta, self.n_rho = n_theta, n_rho
        self.max_peaks = max_peaks
        self.export_acc = export_acc
        flags = (HOUGH_FLAG_EXPORT_ACC if export_acc else 0) | (HOUGH_FLAG_FP64 if fp64 else 0)
        self.ctx = hough_create(self.geometry, n_theta, n_rho, vote_threshold, assoc_tol_bins,
                                max_peaks, flags)

    def close(self):
        if self.ctx:
            hough_destroy(self.ctx)
            self.ctx = None

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass

    def alloc_outputs(self, n_windows: int, n_hits: int, device="cuda", pin=False) -> dict:
        import torch
        kw = dict(device=device)
        if device == "cpu" and pin:
            kw["pin_memory"] = True
        out = dict(
            peaks=torch.zeros((n_windows, max(self.max_peaks, 1), 4), dtype=torch.int32, **kw),
            n_peaks=torch.zeros(n_windows, dtype=torch.int32, **kw),
            n_found=torch.zeros(n_windows, dtype=torch.int32, **kw),
            hit_track=torch.zeros(max(n_hits, 1), dtype=torch.int32, **kw),
            track_hits=torch.zeros(max(n_hits, 1), dtype=torch.int32, **kw),
            window_status=torch.zeros(n_windows, dtype=torch.int32, **kw),
        )
        if self.export_acc:
            out["acc"] = torch.zeros((n_windows, self.n_theta, self.n_rho), dtype=torch.int32, **kw)
        return out

    @staticmethod
    def hits_struct(hits: dict) -> hough_hits:
        if "vane" in hits:
            return make_hits(vane=hits["vane"], strip=hits["strip"], n_hits=hits["vane"].numel()
                             if hasattr(hits["vane"], "numel") else len(hits["vane"]))
        return make_hits(phi_q=hits["phi_q"], z_q=hits["z_q"], n_hits=hits["phi_q"].numel()
                         if hasattr(hits["phi_q"], "numel") else len(hits["phi_q"]))

    def _checked(self, hits: dict, offsets, out: dict | None, cuda: bool) -> tuple:
        """Check the buffers of a find call; returns (n_windows, n_hits, out)."""
        import torch
        n_hits = _check_hits(hits, cuda)
        _check_buf(offsets, torch.int64, 1, cuda, "offsets")
        n_windows = int(offsets.numel()) - 1
        if out is None:
            out = self.alloc_outputs(n_windows, n_hits, device="cuda" if cuda else "cpu", pin=not cuda)
        _check_outputs(out, n_windows, n_hits, self.max_peaks,
                       (self.n_theta, self.n_rho) if self.export_acc else None, cuda)
        return n_windows, n_hits, out

    def find(self, hits: dict, offsets, out: dict | None = None, stream=None) -> dict:
        n_windows, _, out = self._checked(hits, offsets, out, cuda=True)
        hough_find(self.ctx, self.hits_struct(hits), offsets, n_windows, make_tracks(out), stream)
        return out

    def accumulate(self, hits: dict, offsets, out: dict | None = None, stream=None) -> dict:
        """Every window's full accumulator (hough_accumulate), no peaks:
        out = dict(acc [n_windows, n_theta, n_rho], window_status [n_windows])."""
        import torch
        n_hits = _check_hits(hits, True)
        _check_buf(offsets, torch.int64, 1, True, "offsets")
        n_windows = int(offsets.numel()) - 1
        if out is None:
            out = dict(acc=torch.empty((n_windows, self.n_theta, self.n_rho), dtype=torch.int32,
                                       device="cuda"),
                       window_status=torch.zeros(max(n_windows, 1), dtype=torch.int32,
                                                 device="cuda"))
        _check_buf(out["acc"], torch.int32, n_windows * self.n_theta * self.n_rho, True, "acc")
        _check_buf(out["window_status"], torch.int32, n_windows, True, "window_status")
        hough_accumulate(self.ctx, self.hits_struct(hits), offsets, n_windows, out["acc"],
                         out["window_status"], stream)
        return out

    def find_host(self, hits: dict, offsets, out: dict | None = None, stream=None) -> dict:
        """End-to-end form: host (ideally pinned) buffers in and out."""
        n_windows, _, out = self._checked(hits, offsets, out, cuda=False)
        hough_find_host(self.ctx, self.hits_struct(hits), offsets, n_windows, make_tracks(out),
                        stream)
        return out

    def extend(self, hits: dict, offsets, found: dict, tol_z: int, out: dict | None = None,
               stream=None) -> dict:
        """Track extension (hough_extend) on the outputs of find() for the same
        hits and windows; returns dict(tracks, ext_track, ext_hits, window_status)."""
        import torch
        n_hits = _check_hits(hits, True)
        _check_buf(offsets, torch.int64, 1, True, "offsets")
        n_windows = int(offsets.numel()) - 1
        _check_outputs(found, n_windows, n_hits, self.max_peaks, None, True)
        hs = self.hits_struct(hits)
        if out is None:
            dev = found["n_peaks"].device
            out = dict(
                tracks=torch.zeros((n_windows, max(self.max_peaks, 1), 4), dtype=torch.int32,
                                   device=dev),
                ext_track=torch.zeros(max(hs.n_hits, 1), dtype=torch.int32, device=dev),
                ext_hits=torch.zeros(max(hs.n_hits, 1), dtype=torch.int32, device=dev),
                window_status=torch.zeros(max(n_windows, 1), dtype=torch.int32, device=dev))
        _check_buf(out.get("tracks"), torch.int32, n_windows * self.max_peaks * 4, True, "tracks")
        _check_buf(out.get("ext_track"), torch.int32, n_hits, True, "ext_track")
        _check_buf(out.get("ext_hits"), torch.int32, n_hits, True, "ext_hits")
        _check_buf(out.get("window_status"), torch.int32, n_windows, True, "window_status")
        hough_extend(self.ctx, hs, offsets, n_windows, make_tracks(found), tol_z, out, stream)
        return out

    def plan(self, hits: dict, offsets, out: dict, stream=None):
        n_windows, _, out = self._checked(hits, offsets, out, cuda=True)
        return hough_plan_create(self.ctx, self.hits_struct(hits), offsets, n_windows,
                                 make_tracks(out), stream)

    def time_slice(self, t, hits: dict, t0: int, step: int, length: int, n_windows: int,
                   stream=None) -> dict:
        """Cut a time-ordered hit stream (device tensors) into overlapping
        windows; returns dict(hits=..., offsets, index, status, capacity) ready
        for find()."""
        import torch
        _check_buf(t, torch.int64, 0, True, "t")
        n = int(t.numel())
        if _check_hits(hits, True) != n:
            raise ValueError("the hits and their times differ in length")
        cap = max(1, n * (length // step))
        raw = "vane" in hits
        a, b = (hits["vane"], hits["strip"]) if raw else (hits["phi_q"], hits["z_q"])
        dev = t.device
        o0 = torch.empty(cap, dtype=torch.int32, device=dev)
        o1 = torch.empty(cap, dtype=torch.int32, device=dev)
        idx = torch.empty(cap, dtype=torch.int64, device=dev)
        offs = torch.empty(n_windows + 1, dtype=torch.int64, device=dev)
        status = torch.empty(1, dtype=torch.int32, device=dev)
        hough_time_slice(self.ctx, t, a, b, t0, step, length, n_windows, o0, o1, idx, offs,
                         status, stream)
        sliced = dict(vane=o0, strip=o1) if raw else dict(phi_q=o0, z_q=o1)
        return dict(hits=sliced, offsets=offs, index=idx, status=status, capacity=cap)

    def autotune(self, hits: dict, offsets, out: dict, iters=3, stream=None) -> dict:
        n_windows, _, out = self._checked(hits, offsets, out, cuda=True)
        return hough_autotune(self.ctx, self.hits_struct(hits), offsets, n_windows,
                              make_tracks(out), iters, stream)


# ------------------------------------------------------------------ serving

def hough_server_clock_ns() -> int:
    return int(load().hough_server_clock_ns())


class Server:
    """The request loop of libhough over one Finder's context (host buffers).

    submit() queues one time slice (numpy arrays in host memory, ideally
    pinned) and returns a ticket; the arrays are held here until the request
    is delivered by wait() or poll().  While the server exists it owns the
    Finder's context.
    """

    def __init__(self, finder: "Finder", n_slots=4, slot_windows=4096, slot_hits=1 << 20,
                 max_queued=4096, raw_hits=True, launch=None):
        self.lib = load()
        self.finder = finder
        self.max_peaks = finder.max_peaks
        cfg = hough_server_config(n_slots, 1 if raw_hits else 0, slot_windows, slot_hits,
                                  max_queued, hough_launch(*(launch or (0, 0, 0, 0))))
        h = ctypes.c_void_p()
        _check(self.lib.hough_server_create(finder.ctx, ctypes.byref(cfg), ctypes.byref(h)),
               "hough_server_create")
        self.h = h
        self.raw_hits = raw_hits
        self._held = {}

    def submit(self, in0, in1, offsets, out: dict, arrival_ns: int = 0) -> int:
        """Queue windows (in0/in1: vane/strip or phi_q/z_q, int32; offsets int64
        starting at 0); results go to the host arrays of `out` (as Finder
        outputs).  Raises HoughError (code HOUGH_ERR_BUSY when the queue is full)."""
        offsets = np.ascontiguousarray(offsets, np.int64)
        n_windows = len(offsets) - 1
        n_hits = int(offsets[-1]) if n_windows >= 0 else 0
        # the worker reads the inputs and writes the outputs through these
        # pointers: check types and sizes here (the library checks the offsets)
        for name, x, dt, n in [("in0", in0, np.int32, n_hits), ("in1", in1, np.int32, n_hits),
                               ("n_peaks", out.get("n_peaks"), np.int32, n_windows),
                               ("window_status", out.get("window_status"), np.int32, n_windows),
                               ("hit_track", out.get("hit_track"), np.int32, n_hits),
                               ("track_hits", out.get("track_hits"), np.int32, n_hits),
                               ("peaks", out.get("peaks"), np.int32,
                                n_windows * self.finder.max_peaks * 4)]:
            _check_host(x, dt, n, name)
        if out.get("n_found") is not None:
            _check_host(out["n_found"], np.int32, n_windows, "n_found")
        req = hough_request(_ptr(in0), _ptr(in1), _ptr(offsets), n_windows,
                            make_tracks(out), int(arrival_ns))
        t = ctypes.c_uint64()
        _check(self.lib.hough_server_submit(self.h, ctypes.byref(req), ctypes.byref(t)),
               "hough_server_submit")
        self._held[int(t.value)] = (in0, in1, offsets, out)
        return int(t.value)

    def wait(self, ticket: int, timeout_ms: int = -1) -> dict:
        r = hough_request_result()
        _check(self.lib.hough_server_wait(self.h, ticket, timeout_ms, ctypes.byref(r)),
               "hough_server_wait")
        self._held.pop(ticket, None)
        return r.as_dict()

    def poll(self, cap: int = 4096) -> list:
        buf = (hough_request_result * cap)()
        n = ctypes.c_int64()
        _check(self.lib.hough_server_poll(self.h, buf, cap, ctypes.byref(n)), "hough_server_poll")
        out = [buf[i].as_dict() for i in range(n.value)]
        for r in out:
            self._held.pop(r["ticket"], None)
        return out

    def drain(self, timeout_ms: int = -1) -> None:
        _check(self.lib.hough_server_drain(self.h, timeout_ms), "hough_server_drain")

    def stats(self) -> dict:
        st = hough_server_stats()
        _check(self.lib.hough_server_get_stats(self.h, ctypes.byref(st)), "hough_server_get_stats")
        return st.as_dict()

    def close(self) -> None:
        if self.h:
            self.lib.hough_server_destroy(self.h)
            self.h = None
            self._held.clear()

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass
