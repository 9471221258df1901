"""Pins of the oracle's FP64 variant of the find (bins from Eq. (1) in
double precision with the Section 5 binning, instead of the fixed-point
tables): its accumulator against a histogram of an independent numpy
evaluation of Eq. (1), the within-one-bin agreement with the fixed-point
find, and the rest of the find unchanged."""
import math

import numpy as np
import pytest

import oracle
from paper_2511_02742_gb300 import synth

G = synth.GEOMETRY


def numpy_bins(n_theta, n_rho, phi_q, z_q, geom=G):
    theta = (np.arange(n_theta) + 0.5) * (math.pi / n_theta)
    phi = np.asarray(phi_q, np.float64) / geom["phi_u_per_deg"]
    z = np.asarray(z_q, np.float64) / geom["z_u_per_mm"]
    rho = phi[:, None] * np.cos(theta)[None, :] + z[:, None] * np.sin(theta)[None, :]
    x = (rho - geom["rho_min"]) / ((geom["rho_max"] - geom["rho_min"]) / n_rho)
    return x


@pytest.mark.parametrize("n_theta,n_rho,rho_half", [(180, 1000, 500.0), (256, 256, 500.0),
                                                    (97, 332, 500.0), (128, 256, 250.0)])
def test_fp64_accumulator_is_the_histogram_of_eq1(n_theta, n_rho, rho_half):
    """Random hits of the box plus hits outside it (which do not vote); with a
    narrower rho range some votes fall below rho_min and are dropped."""
    geom = dict(G, rho_min=-rho_half, rho_max=rho_half)
    rng = np.random.default_rng(21)
    phi = rng.integers(0, 360 * 200, 300).astype(np.int32)
    z = rng.integers(-38912, 38912 + 1, 300).astype(np.int32)
    phi[:10] = 72000 + rng.integers(0, 500, 10)                # outside the box
    z[10:20] = 39000 + rng.integers(0, 500, 10)
    valid = np.ones(300, bool)
    valid[:20] = False
    x = numpy_bins(n_theta, n_rho, phi, z, geom)[valid]
    frac = x - np.floor(x)
    assert ((frac > 1e-9) & (frac < 1 - 1e-9)).all()     # no value on an edge
    b = np.floor(x).astype(np.int64)
    ref = np.zeros((n_theta, n_rho), np.int64)
    t = np.broadcast_to(np.arange(n_theta)[None, :], b.shape)
    ok = (b >= 0) & (b < n_rho)
    np.add.at(ref, (t[ok], b[ok]), 1)
    r = oracle.find_window(geom, n_theta, n_rho, phi, z, fp64=True)
    np.testing.assert_array_equal(r["acc"], ref)
    assert r["n_dropped"] == int((~ok).sum())
    if rho_half < 409:
        assert (x < 0).any()                # votes below rho_min: floor, not truncation


def test_fp64_association_uses_the_fp64_bins():
    """Each hit goes to the first peak (in order) whose row's FP64 bin, from
    the independent numpy evaluation, is within one bin of the peak's."""
    w = synth.generate(60, ("poisson", 10, 1, 40), (100.0, 300.0), 0.02, seed=26)
    phi, z = oracle.encode(G, w.vane, w.strip)
    r = oracle.find_batch(G, 256, 256, phi, z, w.offsets, fp64=True)
    checked = 0
    for k in range(w.n_windows):
        s = w.window(k)
        x = numpy_bins(256, 256, phi[s], z[s])
        frac = x - np.floor(x)
        if not ((frac > 1e-9) & (frac < 1 - 1e-9)).all():
            continue
        b = np.floor(x).astype(np.int64)
        pk = r["peaks"][k][:r["n_peaks"][k]]
        for h in range(s.stop - s.start):
            m = np.flatnonzero(np.abs(b[h, pk["theta"].astype(int)] - pk["rho"].astype(int)) <= 1)
            assert r["hit_track"][s][h] == (m[0] if len(m) else -1)
            checked += 1
    assert checked > 3000


def test_fp64_and_fixed_accumulators_differ_by_votes_moved_one_bin():
    """Every vote lands within one rho bin of its fixed-point bin, so the FP64
    count of a bin never exceeds the fixed counts of it and its two rho
    neighbours, and the totals are equal."""
    w = synth.workload("plain", n_windows=20, seed=22)
    phi, z = oracle.encode(G, w.vane, w.strip)
    a = oracle.find_batch(G, 512, 512, phi, z, w.offsets, export_acc=True)
    b = oracle.find_batch(G, 512, 512, phi, z, w.offsets, export_acc=True, fp64=True)
    fa, fb = a["acc"].astype(np.int64), b["acc"].astype(np.int64)
    assert (fa.sum(axis=(1, 2)) == fb.sum(axis=(1, 2))).all()
    pad = np.pad(fa, ((0, 0), (0, 0), (1, 1)))
    assert (fb <= pad[:, :, :-2] + pad[:, :, 1:-1] + pad[:, :, 2:]).all()
    assert (fa != fb).any()                  # the two definitions do differ somewhere


@pytest.mark.parametrize("tracks,p_range,noise,seed", [
    (1, (200.0, 300.0), 0.0, 23),
    (1, (100.0, 300.0), 0.0, 24),
    (("poisson", 10, 1, 40), (100.0, 300.0), 0.02, 25),
])
def test_top_peak_agrees_within_one_bin(tracks, p_range, noise, seed):
    """The FP64 top peak lies within one bin (theta and rho) of a fixed-point
    peak holding at least the fixed-point top count minus one, in every
    window whose top peak has at least 10 votes.  (A vote moves by at most
    one rho bin, so a count changes by at most the votes moved; along the
    ridge of a line several bins hold nearly the top count, and one moved
    vote can make another of them the maximum.)"""
    w = synth.generate(300, tracks, p_range, noise, seed=seed)
    phi, z = oracle.encode(G, w.vane, w.strip)
    a = oracle.find_batch(G, 512, 512, phi, z, w.offsets)
    b = oracle.find_batch(G, 512, 512, phi, z, w.offsets, fp64=True)
    n = same = 0
    for k in range(w.n_windows):
        if a["n_peaks"][k] == 0 or a["peaks"][k][0]["votes"] < 10:
            continue
        n += 1
        pa = a["peaks"][k][:a["n_peaks"][k]]
        pb = b["peaks"][k][0]
        near = pa[pa["votes"] >= int(pa[0]["votes"]) - 1]
        ok = (np.abs(near["theta"].astype(int) - int(pb["theta"])) <= 1) & \
             (np.abs(near["rho"].astype(int) - int(pb["rho"])) <= 1)
        assert ok.any(), k
        same += bool(ok[0])
    assert n > 80 and same >= 0.95 * n


def test_fp64_flag_changes_only_the_bins():
    """Hits on exact bin centres of one row vote in the same bins either way,
    so the whole find output is the same."""
    w = synth.workload("tiny")
    phi, z = oracle.encode(G, w.vane, w.strip)
    a = oracle.find_batch(G, 256, 256, phi, z, w.offsets)
    b = oracle.find_batch(G, 256, 256, phi, z, w.offsets, fp64=True)
    for key in ("n_peaks", "n_found", "hit_track", "track_hits", "status"):
        np.testing.assert_array_equal(a[key], b[key])
