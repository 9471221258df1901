"""The iterative highest-bin kernel against the oracle, bit-exact: tracks
(theta, rho, votes, n_hits), their number and every hit's track."""
import numpy as np
import pytest

import oracle
from paper_2511_02742_gb300 import synth

pytestmark = pytest.mark.gpu
G = synth.GEOMETRY


def _gpu(hough, w, n_theta, n_rho, max_tracks=64):
    import torch
    f = hough.Finder(n_theta, n_rho)
    hits = dict(vane=torch.from_numpy(w.vane).cuda(), strip=torch.from_numpy(w.strip).cuda())
    tr = torch.full((w.n_windows, max_tracks, 4), -7, dtype=torch.int32, device="cuda")
    nt = torch.full((w.n_windows,), -7, dtype=torch.int32, device="cuda")
    ht = torch.full((max(w.n_hits, 1),), -7, dtype=torch.int32, device="cuda")
    st = torch.zeros(w.n_windows, dtype=torch.int32, device="cuda")
    hough.hough_find_iterative(f.ctx, f.hits_struct(hits), torch.from_numpy(w.offsets).cuda(),
                               w.n_windows, max_tracks, tr, nt, ht, st)
    torch.cuda.synchronize()
    f.close()
    return (tr.cpu().numpy().view(hough.ITER_DTYPE).reshape(w.n_windows, max_tracks),
            nt.cpu().numpy(), ht.cpu().numpy()[:w.n_hits], st.cpu().numpy())


def _check(hough, w, n_theta, n_rho, max_tracks=64):
    tr, nt, ht, st = _gpu(hough, w, n_theta, n_rho, max_tracks)
    phi, z = oracle.encode(G, w.vane, w.strip)
    rtr, rnt, rht = oracle.iterative(G, n_theta, n_rho, phi, z, w.offsets, max_tracks=max_tracks)
    np.testing.assert_array_equal(nt, rnt)
    for k in range(w.n_windows):
        np.testing.assert_array_equal(tr[k][:nt[k]], rtr[k][:nt[k]], err_msg=str(k))
    np.testing.assert_array_equal(ht, rht)
    assert (st == 0).all()


def test_plain_and_tiny(hough):
    _check(hough, synth.workload("plain", n_windows=60, seed=31), 512, 512)
    _check(hough, synth.workload("tiny"), 256, 256)


def test_uneven_windows_other_shapes_and_truncation(hough):
    w = synth.generate(80, ("poisson", 10, 0, 40), (100.0, 300.0), 0.02, seed=32)
    _check(hough, w, 512, 512)
    _check(hough, w, 180, 1000, max_tracks=3)
    _check(hough, synth.workload("high_pileup", n_windows=4, seed=33), 1024, 1024)


@pytest.mark.parametrize("th1,r1,th2,r2", [(30, 0, 120, -175), (60, -100, 150, -200),
                                           (20, 50, 100, -200), (70, -125, 110, -200)])
def test_equal_lines_in_different_tiles(hough, th1, r1, th2, r2):
    """Two lines of 12 hits each whose highest bins lie in different theta
    tiles with equal counts: the first bin in row-major order is taken first,
    whatever order the tiles are visited in; a third, shorter line and noise
    around them."""
    a = synth.line_window(th1, r1, vanes=range(0, 12))
    b = synth.line_window(th2, r2, vanes=range(20, 32))
    c = synth.line_window(90.0, 30.0, vanes=range(33, 39))
    rng = np.random.default_rng(th1)
    noise_v = rng.integers(0, 40, 8).astype(np.int32)
    noise_s = rng.integers(0, 2048, 8).astype(np.int32)
    for order in (0, 1):
        parts = [(a.vane, a.strip), (b.vane, b.strip)][::1 if order == 0 else -1]
        vane = np.concatenate([parts[0][0], parts[1][0], c.vane, noise_v])
        strip = np.concatenate([parts[0][1], parts[1][1], c.strip, noise_s])
        w = synth.Windows(vane, strip, np.array([0, len(vane)], np.int64),
                          np.zeros(len(vane), np.int32), np.zeros(len(vane)), np.zeros((1, 4)),
                          np.array([0, 1], np.int64))
        _check(hough, w, 512, 512)
        _check(hough, w, 1024, 1024)
