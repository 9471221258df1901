"""Pins of the oracle's coarse-to-fine search (the paper's two-stage GPU
method: an 18 x 100 coarse histogram, then a 10 x 10 fine histogram of the
180 x 1000 grid around its maximum)."""
import numpy as np
import pytest

import oracle
from paper_2511_02742_gb300 import synth

G = synth.GEOMETRY


def _run(w):
    phi, z = oracle.encode(G, w.vane, w.strip)
    return oracle.coarse_fine(G, phi, z, w.offsets), phi, z


@pytest.mark.parametrize("theta_deg,fine_rho_bin", [(84.5, 505), (95.5, 495), (104.5, 503)])
def test_single_line_closed_form(theta_deg, fine_rho_bin):
    """Hits on the line through the centre of fine bin (t, b) of the 180 x 1000
    grid, half a degree from a coarse row's centre: the coarse maximum is the
    coarse bin containing it and the fine maximum is that bin, holding every
    hit, all of them seeds.  (Lines far from every coarse centre spread over
    several coarse rho bins: the method's own limit.)"""
    rho = -500.0 + fine_rho_bin + 0.5
    w = synth.line_window(theta_deg, rho)
    (res, ht), _, _ = _run(w)
    r = res[0]
    t = int(theta_deg)                               # centre (t + 0.5) degrees
    assert (r["coarse_theta"], r["coarse_rho"]) == (t // 10, fine_rho_bin // 10)
    assert (r["fine_theta"], r["fine_rho"]) == (t, fine_rho_bin)
    assert r["fine_votes"] == w.n_hits and r["coarse_votes"] == w.n_hits
    assert r["found"] == 1 and r["n_seeds"] == w.n_hits and (ht == 0).all()
    assert w.n_hits >= 30


def test_agrees_with_the_full_histograms():
    """The coarse maximum is the maximum of the 18 x 100 accumulator and the
    fine result is the maximum of the 180 x 1000 accumulator restricted to
    the coarse bin's 10 x 10 block (first in row-major order on ties)."""
    w = synth.workload("plain", n_windows=25, seed=9)
    (res, ht), phi, z = _run(w)
    for k in range(w.n_windows):
        sl = w.window(k)
        acc_c, _ = oracle.vote(G, 18, 100, phi[sl], z[sl])
        acc_f, _ = oracle.vote(G, 180, 1000, phi[sl], z[sl])
        r = res[k]
        ci = int(np.argmax(acc_c))                   # first maximum, row-major
        assert (r["coarse_theta"], r["coarse_rho"]) == divmod(ci, 100)
        assert r["coarse_votes"] == acc_c.max()
        if r["coarse_votes"] < 5:
            assert r["found"] == 0
            continue
        tc, bc = divmod(ci, 100)
        block = acc_f[tc * 10:tc * 10 + 10, bc * 10:bc * 10 + 10]
        fi = int(np.argmax(block))
        assert (r["fine_theta"], r["fine_rho"]) == (tc * 10 + fi // 10, bc * 10 + fi % 10)
        assert r["fine_votes"] == block.max()
        assert r["found"] == int(block.max() >= 5)


def test_seeds_are_the_hits_on_the_line():
    w = synth.workload("plain", n_windows=25, seed=10)
    (res, ht), phi, z = _run(w)
    for k in range(w.n_windows):
        sl = w.window(k)
        r = res[k]
        if not r["found"]:
            assert (ht[sl] < 0).all()
            continue
        bins = oracle.bins_fixed(G, 180, 1000, phi[sl], z[sl])[:, r["fine_theta"]]
        on = np.abs(bins - r["fine_rho"]) <= 1
        np.testing.assert_array_equal(ht[sl] == 0, on)
        assert r["n_seeds"] == on.sum()


def test_empty_window_and_rejected_hits():
    w = synth.Windows(np.array([99, 3], np.int32), np.array([5, 99999], np.int32),
                      np.array([0, 0, 2], np.int64), np.zeros(2, np.int32), np.zeros(2),
                      np.zeros((1, 4)), np.array([0, 1], np.int64))
    (res, ht), _, _ = _run(w)
    assert res[0]["found"] == 0 and res[0]["coarse_votes"] == 0
    assert list(ht) == [-2, -2]
