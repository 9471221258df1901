"""Pins of the oracle's iterative highest-bin search (the literal reading of
the paper's peak step, repeated: highest bin, its line's hits, remove, vote
again)."""
import math

import numpy as np
import pytest

import oracle
from paper_2511_02742_gb300 import synth

G = synth.GEOMETRY


def _line_hits(th_deg, rho, vanes):
    """Fixed-point hits exactly (to 1/200 mm) on phi cos th + z sin th = rho."""
    th = math.radians(th_deg)
    phi_q, z_q = [], []
    for k in vanes:
        z = (rho - 9.0 * k * math.cos(th)) / math.sin(th)
        phi_q.append(1800 * k)
        z_q.append(int(round(z * 200.0)))
    return np.array(phi_q, np.int32), np.array(z_q, np.int32)


def _centred(t, b, n_theta=512, n_rho=512):
    return (t + 0.5) * 180.0 / n_theta, -500.0 + (b + 0.5) * 1000.0 / n_rho


def test_two_lines_are_taken_in_order_of_size():
    """A 30-hit line and a 12-hit line: track 0 is the larger one at its
    bin with all of its hits; then the smaller one (within one bin: its few
    sinusoids meet nearly in parallel, so neighbouring rows can tie and the
    first in row-major order is taken); then nothing."""
    ta, ra = _centred(150, 260)
    tb, rb = _centred(330, 240)
    pa, za = _line_hits(ta, ra, range(0, 30))
    pb, zb = _line_hits(tb, rb, range(5, 17))
    phi = np.concatenate([pa, pb])
    z = np.concatenate([za, zb])
    tr, nt, ht = oracle.iterative(G, 512, 512, phi, z, np.array([0, len(phi)]))
    assert nt[0] == 2
    assert (tr[0][0]["theta"], tr[0][0]["rho"], tr[0][0]["votes"]) == (150, 260, 30)
    assert abs(int(tr[0][1]["theta"]) - 330) <= 1 and abs(int(tr[0][1]["rho"]) - 240) <= 1
    assert tr[0][1]["votes"] == 12
    assert (ht[:30] == 0).all() and (ht[30:] == 1).all()
    assert tr[0][0]["n_hits"] == 30 and tr[0][1]["n_hits"] == 12


def test_against_the_full_accumulator():
    """Track 0 is the first maximum of the whole accumulator; each later
    track is the first maximum of the accumulator of the hits left over; its
    hits are those within one bin of it in its row; votes never increase."""
    w = synth.workload("plain", n_windows=12, seed=21)
    phi, z = oracle.encode(G, w.vane, w.strip)
    tr, nt, ht = oracle.iterative(G, 512, 512, phi, z, w.offsets)
    for k in range(w.n_windows):
        sl = w.window(k)
        p, q, h = phi[sl], z[sl], ht[sl]
        left = np.ones(len(p), bool)
        prev = None
        for j in range(nt[k]):
            acc, _ = oracle.vote(G, 512, 512, p[left], q[left])
            t, b = divmod(int(np.argmax(acc)), 512)
            r = tr[k][j]
            assert (r["theta"], r["rho"], r["votes"]) == (t, b, acc.max())
            assert prev is None or r["votes"] <= prev
            assert r["votes"] >= 5
            prev = r["votes"]
            bins = oracle.bins_fixed(G, 512, 512, p, q)[:, t]
            mine = left & (np.abs(bins - b) <= 1)
            np.testing.assert_array_equal(h == j, mine)
            assert r["n_hits"] == mine.sum() >= r["votes"]
            left &= ~mine
        acc, _ = oracle.vote(G, 512, 512, p[left], q[left])
        assert acc.max() < 5 or nt[k] == 64
        assert (h[left] == -1).all()


def test_max_tracks_truncates():
    w = synth.workload("plain", n_windows=6, seed=22)
    phi, z = oracle.encode(G, w.vane, w.strip)
    full, nf, _ = oracle.iterative(G, 512, 512, phi, z, w.offsets)
    two, n2, ht2 = oracle.iterative(G, 512, 512, phi, z, w.offsets, max_tracks=2)
    np.testing.assert_array_equal(n2, np.minimum(nf, 2))
    for k in range(w.n_windows):
        np.testing.assert_array_equal(two[k][:n2[k]], full[k][:n2[k]])
    assert ht2.max() <= 1
