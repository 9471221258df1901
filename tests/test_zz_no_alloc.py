"""The allocation-free entry point (hough_find_noalloc) against hough_find.

Callers that cannot call cudaMalloc (and so cannot create a context) use
hough_find_noalloc, which keeps the kernel's scheduling counters and tables in
a fixed device array of the library.  Its results must be the same bits as the
context-based entry point's, on two calls in a row: the second call reuses the
array the first one left behind (other shape, other windows), so a counter
that was not cleared or a stale table would show up there.
"""
import contextlib
import ctypes

import numpy as np
import pytest

from paper_2511_02742_gb300 import synth

pytestmark = pytest.mark.gpu


def _inputs(hough, w):
    import torch
    hits = dict(vane=torch.from_numpy(w.vane).cuda(), strip=torch.from_numpy(w.strip).cuda())
    offs = torch.from_numpy(w.offsets).cuda()
    return hits, offs


def _numpy(out, n_hits):
    r = {k: v.cpu().numpy() for k, v in out.items()}
    r["hit_track"] = r["hit_track"][:n_hits]
    r["track_hits"] = r["track_hits"][:n_hits]
    return r


@pytest.mark.parametrize("first,second", [((512, 512, 7), (256, 256, 8)),
                                          ((1024, 1024, 9), (512, 512, 10))])
def test_noalloc_matches_hough_find_twice_in_a_row(first, second):
    import torch
    from paper_2511_02742_gb300 import hough
    hough.load()
    for n_theta, n_rho, seed in (first, second):
        w = synth.generate(200, ("poisson", 10, 1, 40), (100.0, 300.0), 0.02, seed=seed)
        hits, offs = _inputs(hough, w)
        f = hough.Finder(n_theta, n_rho)
        ref = f.find(hits, offs)
        out = f.alloc_outputs(w.n_windows, w.n_hits)
        for v in out.values():
            v.fill_(-7)
        hough.hough_find_noalloc(synth.GEOMETRY, n_theta, n_rho, f.hits_struct(hits), offs,
                                 w.n_windows, hough.make_tracks(out))
        torch.cuda.synchronize()
        a, b = _numpy(ref, w.n_hits), _numpy(out, w.n_hits)
        for k in ("n_peaks", "n_found", "window_status", "hit_track", "track_hits"):
            np.testing.assert_array_equal(b[k], a[k], err_msg=k)
        pa, pb = hough.decode_peaks(ref["peaks"]), hough.decode_peaks(out["peaks"])
        for k in range(w.n_windows):
            n = int(a["n_peaks"][k])
            np.testing.assert_array_equal(pb[k][:n], pa[k][:n])
        f.close()


def test_noalloc_rejects_sizes_beyond_its_array():
    from paper_2511_02742_gb300 import hough
    lib = hough.load()
    g = hough.make_geometry(synth.GEOMETRY)
    th = hough.hough_thresholds(5, 1, 64, 0)
    hits = hough.hough_hits(None, None, None, None, 0)
    tracks = hough.hough_tracks()
    rc = lib.hough_find_noalloc(ctypes.byref(g), hough.HOUGH_NOALLOC_MAX_THETA + 1, 512,
                                ctypes.byref(th), ctypes.byref(hits), None, 0,
                                ctypes.byref(tracks), None)
    assert rc == -5          # HOUGH_ERR_UNSUPPORTED_SHAPE


def test_noalloc_export_on_a_side_stream_at_the_row_limit():
    """n_theta at the array's exact limit (HOUGH_NOALLOC_MAX_THETA rows of
    tables) with every accumulator exported, on a side stream; then another
    shape without export on the default stream.  Both calls equal the oracle
    (accumulators included) and hough_find, bit for bit."""
    import torch
    from paper_2511_02742_gb300 import hough
    from parity_helpers import assert_batch_equal, oracle_run, to_numpy
    hough.load()
    side = torch.cuda.Stream()
    cases = [(hough.HOUGH_NOALLOC_MAX_THETA, 8, True, side, 21), (256, 256, False, None, 22)]
    for n_theta, n_rho, export, stream, seed in cases:
        w = synth.generate(30, ("poisson", 6, 1, 20), (100.0, 300.0), 0.02, seed=seed)
        hits, offs = _inputs(hough, w)
        f = hough.Finder(n_theta, n_rho, export_acc=export)
        out = f.alloc_outputs(w.n_windows, w.n_hits)
        for v in out.values():
            v.fill_(-7)
        torch.cuda.synchronize()
        flags = hough.HOUGH_FLAG_EXPORT_ACC if export else 0
        with torch.cuda.stream(stream) if stream is not None else contextlib.nullcontext():
            hough.hough_find_noalloc(synth.GEOMETRY, n_theta, n_rho, f.hits_struct(hits), offs,
                                     w.n_windows, hough.make_tracks(out), flags=flags,
                                     stream=torch.cuda.current_stream())
        torch.cuda.synchronize()
        got = to_numpy(out, w.n_hits)
        ref = oracle_run(w, n_theta, n_rho, export=export)
        assert_batch_equal(got, ref, w, check_acc=export)
        viaf = to_numpy(f.find(hits, offs), w.n_hits)
        torch.cuda.synchronize()
        for k in ("n_peaks", "n_found", "status", "hit_track", "track_hits") + \
                (("acc",) if export else ()):
            np.testing.assert_array_equal(got[k], viaf[k], err_msg=k)
        f.close()


def test_noalloc_refuses_a_capturing_stream():
    """Each call copies its tables from host memory, which a stream capturing
    a graph cannot take: such a call is refused with INVALID_ARG before
    anything is enqueued, and the capture goes on (the graph replays)."""
    import torch
    from paper_2511_02742_gb300 import hough
    w = synth.generate(20, ("poisson", 5, 1, 20), (100.0, 300.0), 0.02, seed=31)
    hits, offs = _inputs(hough, w)
    f = hough.Finder(256, 256)
    out = f.alloc_outputs(w.n_windows, w.n_hits)
    # an ordinary call first: the device's set-up happens outside any capture
    hough.hough_find_noalloc(synth.GEOMETRY, 256, 256, f.hits_struct(hits), offs, w.n_windows,
                             hough.make_tracks(out))
    torch.cuda.synchronize()
    x = torch.zeros(4, device="cuda")
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, capture_error_mode="thread_local"):
        x.add_(1)
        with pytest.raises(hough.HoughError) as e:
            hough.hough_find_noalloc(synth.GEOMETRY, 256, 256, f.hits_struct(hits), offs,
                                     w.n_windows, hough.make_tracks(out),
                                     stream=torch.cuda.current_stream())
        assert e.value.code == hough.HOUGH_ERR_INVALID_ARG
        x.add_(1)
    g.replay()
    torch.cuda.synchronize()
    assert x.tolist() == [2.0, 2.0, 2.0, 2.0]
    f.close()
