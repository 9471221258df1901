"""The allocation-free entry point (hough_find_noalloc) against hough_find.

Callers that cannot call cudaMalloc (and so cannot create a context) use
hough_find_noalloc, which keeps the kernel's scheduling counters and tables in
a fixed device array of the library.  Its results must be the same bits as the
context-based entry point's, on two calls in a row: the second call reuses the
array the first one left behind (other shape, other windows), so a counter
that was not cleared or a stale table would show up there.
"""
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
