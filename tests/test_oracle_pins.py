"""Pins of the CPU oracle against facts that do not come from the oracle itself.

Each test names the passage of the paper it rests on.  The oracle is the
reference for the CUDA parity tests, so a mistake in it (a dropped term, a
wrong sign or index, a transposed operand, a wrong tie-break) must fail here.
"""
import math

import numpy as np
import pytest

import oracle
from golden_io import geometry_facts, peak_cases
from paper_2511_02742_gb300 import synth

G = synth.GEOMETRY
SHAPES = [(180, 1000), (256, 256), (512, 512), (1024, 1024), (97, 334)]


def fp64_rho_bins(geom, n_theta, n_rho, phi_q, z_q):
    """Eq. (1) in double precision, with the Section 5 binning: returns the
    continuous bin coordinate (rho - rho_min)/drho for every (hit, theta)."""
    theta = (np.arange(n_theta) + 0.5) * (math.pi / n_theta)
    phi = np.asarray(phi_q, np.float64) / geom["phi_u_per_deg"]
    z = np.asarray(z_q, np.float64) / geom["z_u_per_mm"]
    rho = phi[:, None] * np.cos(theta)[None, :] + z[:, None] * np.sin(theta)[None, :]
    drho = (geom["rho_max"] - geom["rho_min"]) / n_rho
    return (rho - geom["rho_min"]) / drho


def random_valid_hits(rng, n, any_phi=False):
    if any_phi:
        phi = rng.integers(0, 360 * 200, n).astype(np.int32)
    else:
        phi = (rng.integers(0, 40, n) * 1800).astype(np.int32)
    z = rng.integers(-38912, 38912 + 1, n).astype(np.int32)
    return phi, z


# --------------------------------------------------------------- geometry ---

def test_geometry_matches_section2():
    """Section 2: 40 vanes x 16 sensors, 2 blocks x 512 strips at 190 um,
    97.28 mm sensors, |z| <= 200 mm, 16,384 strips per vane, 655k in total."""
    f = geometry_facts()
    strips_per_vane = f["sensors_per_vane"] * f["strip_blocks_per_sensor"] * f["strips_per_block"]
    assert strips_per_vane == f["strips_per_vane"]
    assert abs(f["n_vanes"] * strips_per_vane - f["strips_total_approx"]) / 655000 < 0.01
    assert abs(f["strips_per_block"] * f["strip_pitch_mm"] - f["sensor_side_mm"]) < 1e-9
    # The reading used here: 4 Z-sensors along z, each 512 strips of 0.19 mm.
    assert G["n_vanes"] == f["n_vanes"]
    assert G["n_z_strips"] == 4 * f["strips_per_block"]
    assert G["z_pitch_u"] == round(f["strip_pitch_mm"] * G["z_u_per_mm"])
    assert abs(G["z_pitch_u"] / G["z_u_per_mm"] - f["strip_pitch_mm"]) < 1e-12
    span = G["n_z_strips"] * G["z_pitch_u"] / G["z_u_per_mm"]
    assert abs(span - 4 * f["sensor_side_mm"]) < 1e-9
    assert span / 2 <= f["z_half_range_mm"]


def test_encoding_phi_is_vane_angle_and_z_is_strip_centre():
    """Section 2 (radial vanes) and Section 5 (phi = atan(y/x)): every point on
    vane k has phi = 9 deg * k; a z strip j measures the centre of the strip."""
    vane = np.repeat(np.arange(40, dtype=np.int32), 3)
    strip = np.tile(np.array([0, 1023, 2047], np.int32), 40)
    phi, z = oracle.encode(G, vane, strip)
    # phi from the vane's azimuth, computed from its direction vector
    ang = np.degrees(np.arctan2(np.sin(np.radians(9.0 * vane)), np.cos(np.radians(9.0 * vane))))
    ang = np.mod(ang, 360.0)
    np.testing.assert_allclose(phi / 200.0, ang, atol=1e-9)
    z_mm = z / 200.0
    centre = synth.Z_MIN_MM + (strip + 0.5) * synth.Z_STRIP_PITCH_MM
    np.testing.assert_allclose(z_mm, centre, atol=1e-9)
    assert np.all(np.abs(z_mm) < 200.0)


# ----------------------------------------------------------------- voting ---

def edge_margin(geom, n_theta, n_rho):
    """Largest possible distance, in bins, between the fixed-point bin
    coordinate and the exact one: each table entry is within 1/2 unit of its
    real factor, so the sum is off by at most (|phi| + |z| + 1) / 2 units of
    2^-K bins over the detector box."""
    k = oracle.tables(geom, n_theta, n_rho)[3]
    phi_max = 360 * geom["phi_u_per_deg"]
    z_max = max(abs(geom["z_min_u"]),
                abs(geom["z_min_u"] + geom["n_z_strips"] * geom["z_pitch_u"]))
    return 0.5 * (phi_max + z_max + 1) / 2.0 ** k + 1e-9


@pytest.mark.parametrize("n_theta,n_rho", SHAPES)
def test_fixed_point_bins_within_one_bin_of_fp64(n_theta, n_rho):
    """Eq. (1) + Section 5 binning: the integer bin from the fixed-point tables
    equals floor of the FP64 rho coordinate, except where that coordinate lies
    within the table-rounding margin of an edge, and is never more than one
    bin away."""
    rng = np.random.default_rng(11)
    phi, z = random_valid_hits(rng, 400, any_phi=True)
    fixed = oracle.bins_fixed(G, n_theta, n_rho, phi, z)
    x = fp64_rho_bins(G, n_theta, n_rho, phi, z)
    ref = np.floor(x).astype(np.int64)
    assert np.abs(fixed - ref).max() <= 1
    eps = edge_margin(G, n_theta, n_rho)
    assert eps < 0.05
    frac = x - np.floor(x)
    safe = (frac > eps) & (frac < 1.0 - eps)
    assert safe.mean() > 0.85
    np.testing.assert_array_equal(fixed[safe], ref[safe])
    # the oracle's own FP64 variant agrees with this independent computation
    fp = oracle.bins_fp64(G, n_theta, n_rho, phi, z)
    safe64 = (frac > 1e-9) & (frac < 1.0 - 1e-9)
    np.testing.assert_array_equal(fp[safe64], ref[safe64])


@pytest.mark.parametrize("n_theta,n_rho", SHAPES)
def test_tables_round_to_nearest(n_theta, n_rho):
    """The fixed-point cos/sin factors of Eq. (1) are rounded to the nearest
    integer: each entry is within half a unit of the real factor
    cos(theta_t) * 2^K * n_rho / (1000 deg * 200 u/deg), and likewise for sin."""
    C, S, D, K = oracle.tables(G, n_theta, n_rho)
    theta = (np.arange(n_theta) + 0.5) * math.pi / n_theta
    scale = 2.0 ** K * n_rho / (1000.0 * 200.0)
    assert np.abs(C - np.cos(theta) * scale).max() <= 0.5 + 1e-6
    assert np.abs(S - np.sin(theta) * scale).max() <= 0.5 + 1e-6
    assert D == (n_rho // 2) << K          # rho_min = -500 is exactly n_rho/2 bins below 0


@pytest.mark.parametrize("n_theta,n_rho", SHAPES + [(64, 4), (512, 1024)])
def test_scale_is_the_largest_that_fits_32_bits(n_theta, n_rho):
    """The scale 2^K is the largest (K <= 24) for which every hit of the
    detector box gives |phi*C + z*S + D| < 2^31 (checked here on a dense grid
    of the box with exact integers), and 2^(K+1) would not fit."""
    C, S, D, K = oracle.tables(G, n_theta, n_rho)
    phi = np.array([0, 1800 * 20, 72000 - 1], dtype=object)
    z = np.array([-38912, 0, 38912], dtype=object)
    vals = [int(p_) * int(c) + int(z_) * int(s_) + D for c, s_ in zip(C, S) for p_ in phi for z_ in z]
    assert max(abs(v) for v in vals) < 2 ** 31
    assert 8 <= K <= 24
    if K < 24:
        # one more bit would overflow somewhere: double the scale by hand
        theta = (np.arange(n_theta) + 0.5) * math.pi / n_theta
        scale = 2.0 ** (K + 1) * n_rho / (1000.0 * 200.0)
        C2 = np.floor(np.abs(np.cos(theta) * scale) + 0.5) * np.sign(np.cos(theta))
        S2 = np.floor(np.abs(np.sin(theta) * scale) + 0.5)
        D2 = (n_rho // 2) << (K + 1)
        big = max(abs(int(p_) * int(c) + int(z_) * int(s_) + D2)
                  for c, s_ in zip(C2, S2) for p_ in (0, 71999) for z_ in (-38912, 38912))
        assert big >= 2 ** 31


def test_fixed_point_edges_of_rho_range():
    """Section 5: rho in [-500, 500) over n_rho bins.  With phi = 0, z = 0,
    rho = 0 sits on the edge between bins n_rho/2 - 1 and n_rho/2 and floors up."""
    for n_theta, n_rho in SHAPES:
        b = oracle.bins_fixed(G, n_theta, n_rho, np.array([0], np.int32), np.array([0], np.int32))
        assert np.all(b == n_rho // 2)


@pytest.mark.parametrize("n_theta,n_rho", [(16, 16), (13, 11), (180, 1000), (64, 96)])
def test_accumulator_matches_fp64_brute_force(n_theta, n_rho):
    """Eq. (1): each hit adds one vote per theta row at its rho bin.  The
    accumulator equals a brute-force FP64 histogram everywhere except in bins
    touched by a vote that lies within 0.02 bin of an edge."""
    rng = np.random.default_rng(n_theta * 1000 + n_rho)
    eps = edge_margin(G, n_theta, n_rho)
    for trial in range(20):
        n = int(rng.integers(0, 9))
        phi, z = random_valid_hits(rng, n, any_phi=bool(trial % 2))
        acc, dropped = oracle.vote(G, n_theta, n_rho, phi, z)
        x = fp64_rho_bins(G, n_theta, n_rho, phi, z)
        b = np.floor(x).astype(np.int64)
        ref = np.zeros((n_theta, n_rho), np.int64)
        near = np.zeros((n_theta, n_rho + 2), bool)
        for h in range(n):
            for t in range(n_theta):
                if 0 <= b[h, t] < n_rho:
                    ref[t, b[h, t]] += 1
                fr = x[h, t] - b[h, t]
                if fr < eps or fr > 1.0 - eps:
                    lo = max(b[h, t] - 1, -1)
                    near[t, lo + 1:b[h, t] + 3] = True
        near = near[:, 1:n_rho + 1]
        np.testing.assert_array_equal(acc[~near], ref[~near])


def test_vote_conservation_and_row_sums():
    """Every valid hit casts exactly one vote per theta row (Eq. (1)): the
    accumulator plus the dropped votes add up to H_valid * n_theta, and each
    row sums to the number of valid hits whose bin in that row is in range."""
    geom = dict(G, rho_min=-150.0, rho_max=120.0)    # narrow range: many votes drop
    rng = np.random.default_rng(5)
    phi, z = random_valid_hits(rng, 300, any_phi=True)
    # a few hits outside the coordinate box are rejected and vote nowhere
    phi = np.concatenate([phi, np.array([72000, -1, 0, 1800], np.int32)])
    z = np.concatenate([z, np.array([0, 0, 38913, -38913], np.int32)])
    for n_theta, n_rho in [(180, 1000), (256, 128)]:
        acc, dropped = oracle.vote(geom, n_theta, n_rho, phi, z)
        assert dropped > 0
        assert acc.sum() + dropped == 300 * n_theta
        x = fp64_rho_bins(geom, n_theta, n_rho, phi[:300], z[:300])
        eps = edge_margin(geom, n_theta, n_rho)
        inside = (x >= eps) & (x < n_rho - eps)
        maybe = (x > -eps) & (x < n_rho + eps)
        rows = acc.sum(axis=1)
        assert np.all(rows >= inside.sum(axis=0))
        assert np.all(rows <= maybe.sum(axis=0))


# --------------------------------------------------------- closed forms ----

LINES = [(30.0, 150.0), (60.0, 100.0), (89.0, -20.0), (100.0, 10.0), (120.0, -80.0),
         (135.0, -150.0), (150.0, -250.0), (75.0, 60.0)]


@pytest.mark.parametrize("n_theta,n_rho", [(180, 1000), (256, 256), (512, 512), (1024, 1024)])
def test_single_line_peaks_at_its_parameters(n_theta, n_rho):
    """Section 4: the sinusoids of collinear (phi, z) points meet at the line's
    (theta, rho).  Hits on the line with theta at a theta-bin centre and rho at
    a rho-bin centre all vote in that bin, and it is the top peak within one
    bin (ties inside a plateau go to the first bin)."""
    drho = 1000.0 / n_rho
    for th_deg, rho in LINES:
        t_star = int(th_deg / (180.0 / n_theta))
        th = (t_star + 0.5) * 180.0 / n_theta
        b_star = int((rho + 500.0) / drho)
        rho_c = -500.0 + (b_star + 0.5) * drho
        w = synth.line_window(th, rho_c)
        n = w.n_hits
        assert n >= 5
        phi, z = oracle.encode(G, w.vane, w.strip)
        r = oracle.find_window(G, n_theta, n_rho, phi, z)
        assert r["acc"][t_star, b_star] == n
        top = r["peaks"][0]
        assert top["votes"] == n
        assert abs(int(top["theta"]) - t_star) <= 1 and abs(int(top["rho"]) - b_star) <= 1
        assert np.all(r["hit_track"] == 0)
        assert r["peaks"][0]["n_hits"] == n


def _tls_line(phi_deg, z_mm):
    """Total-least-squares line n . (phi, z) = rho with n = (cos th, sin th), th in [0, pi)."""
    pts = np.stack([phi_deg, z_mm], axis=1)
    c = pts.mean(axis=0)
    _, _, vt = np.linalg.svd(pts - c)
    nrm = vt[1]
    if nrm[1] < 0 or (nrm[1] == 0 and nrm[0] < 0):
        nrm = -nrm
    th = math.atan2(nrm[1], nrm[0])
    rho = float(nrm @ c)
    resid = (pts - c) @ nrm
    return th, rho, np.abs(resid).max()


def test_helix_peaks_at_true_line():
    """Section 4: a positron helix projects to (nearly) a straight line in the
    phi-z plane.  For generated single tracks whose noise-free crossings lie
    within a quarter of a rho bin of their total-least-squares line, a maximal
    bin of the accumulator lies within one bin of that line's (theta, rho), and
    holds at least half of the hits (at the theta row nearest the line the
    hits spread over less than one rho bin, so over at most two bins)."""
    n_theta = n_rho = 512
    w = synth.generate(2000, 1, (100.0, 300.0), 0.0, seed=3, shuffle=False)
    phi_all, z_all = oracle.encode(G, w.vane, w.strip)
    drho = 1000.0 / n_rho
    dth = math.pi / n_theta
    checked = 0
    for k in range(w.n_windows):
        sl = w.window(k)
        if sl.stop - sl.start < 10:
            continue
        phi_deg = w.vane[sl] * 9.0
        th, rho, res = _tls_line(phi_deg, w.z_mm[sl])
        if res > 0.5 * drho * 0.5:          # half a bin, with margin for digitisation
            continue
        acc, _ = oracle.vote(G, n_theta, n_rho, phi_all[sl], z_all[sl])
        t_fit = int(th / dth)
        b_fit = int(math.floor((rho + 500.0) / drho))
        top = acc.max()
        assert 2 * top >= sl.stop - sl.start
        ts, bs = np.nonzero(acc == top)
        d = np.maximum(np.abs(ts - t_fit), np.abs(bs - b_fit))
        assert d.min() <= 1, (k, t_fit, b_fit, list(zip(ts, bs))[:5])
        checked += 1
    assert checked >= 20


# ----------------------------------------------------------------- peaks ---

@pytest.mark.parametrize("case", list(peak_cases()), ids=lambda c: c["name"])
def test_peaks_hand_built(case):
    """Section 4/5 peak rule on accumulators whose peaks were worked out by hand."""
    pk, found = oracle.peaks(case["acc"], case["T"], case["max_peaks"])
    assert found == case["found"]
    got = [(int(p["theta"]), int(p["rho"]), int(p["votes"])) for p in pk]
    assert got == case["expect"]


def test_peaks_brute_force_random_small():
    """The peak rule, checked bin by bin against a direct restatement of the
    definition on many small random accumulators (including plateaus)."""
    rng = np.random.default_rng(9)
    for _ in range(300):
        nt, nr = int(rng.integers(1, 7)), int(rng.integers(1, 7))
        acc = rng.integers(0, 4, (nt, nr)).astype(np.int32)
        T = int(rng.integers(1, 4))
        expect = []
        for t in range(nt):
            for b in range(nr):
                v = acc[t, b]
                if v < T:
                    continue
                ok = True
                for dt in (-1, 0, 1):
                    for db in (-1, 0, 1):
                        if dt == 0 and db == 0:
                            continue
                        tt, bb = t + dt, b + db
                        if not (0 <= tt < nt and 0 <= bb < nr):
                            continue
                        earlier = (tt, bb) < (t, b)
                        if (earlier and not v > acc[tt, bb]) or (not earlier and not v >= acc[tt, bb]):
                            ok = False
                if ok:
                    expect.append((-int(v), t, b))
        expect.sort()
        k = int(rng.integers(0, 5))
        pk, found = oracle.peaks(acc, T, k)
        assert found == len(expect)
        got = [(-int(p["votes"]), int(p["theta"]), int(p["rho"])) for p in pk]
        assert got == expect[:k]


def test_peaks_are_never_adjacent():
    """Under the tie-break two peaks are never 8-neighbours (one of them would
    have to be both > and <= the other)."""
    rng = np.random.default_rng(1)
    for _ in range(50):
        acc = rng.integers(0, 3, (20, 30)).astype(np.int32)
        pk, found = oracle.peaks(acc, 1, 10000)
        pos = {(int(p["theta"]), int(p["rho"])) for p in pk}
        for t, b in pos:
            for dt in (-1, 0, 1):
                for db in (-1, 0, 1):
                    if (dt or db) and (t + dt, b + db) in pos:
                        raise AssertionError("adjacent peaks")


# ------------------------------------------------------------ association ---

def _line_hits(th_deg, rho, vanes):
    """Fixed-point hits exactly (to 1/200 mm) on phi cos th + z sin th = rho."""
    th = math.radians(th_deg)
    phi_q, z_q = [], []
    for k in vanes:
        phi = 9.0 * k
        z = (rho - phi * math.cos(th)) / math.sin(th)
        phi_q.append(1800 * k)
        z_q.append(int(round(z * 200.0)))
    return np.array(phi_q, np.int32), np.array(z_q, np.int32)


def test_association_two_lines_first_peak_wins():
    """Section 5: seed hits are the hits on the peak's line.  Two lines that
    cross: every hit goes to the first peak (more votes) whose line it lies on
    within one bin; the expectation uses FP64 bins and hand-chosen lines."""
    n_theta = n_rho = 512
    drho = 1000.0 / n_rho
    ta = int(70.0 / (180.0 / n_theta))
    tb = int(115.0 / (180.0 / n_theta))
    tha, thb = (ta + 0.5) * 180.0 / n_theta, (tb + 0.5) * 180.0 / n_theta
    ba, bb = 280, 250
    rhoa, rhob = -500 + (ba + 0.5) * drho, -500 + (bb + 0.5) * drho
    pa, za = _line_hits(tha, rhoa, range(0, 40, 2))      # 20 hits
    pb, zb = _line_hits(thb, rhob, range(1, 40, 3))      # 13 hits
    keep_a = np.abs(za) < 38900
    keep_b = np.abs(zb) < 38900
    # off-line probes near line A at theta_a: +1 bin (inside the tolerance of one
    # bin) and +2 bins (outside), both at a bin centre, on vanes 5 and 33
    probes_phi, probes_z = [], []
    for k, dbins in ((5, 1), (33, 2), (7, -1), (31, -2)):
        ph = 9.0 * k
        rr = rhoa + dbins * drho
        zz = (rr - ph * math.cos(math.radians(tha))) / math.sin(math.radians(tha))
        probes_phi.append(1800 * k)
        probes_z.append(int(round(zz * 200.0)))
    phi = np.concatenate([pa[keep_a], pb[keep_b], np.array(probes_phi, np.int32),
                          np.array([9000], np.int32)])
    z = np.concatenate([za[keep_a], zb[keep_b], np.array(probes_z, np.int32),
                        np.array([30000], np.int32)])
    r = oracle.find_window(G, n_theta, n_rho, phi, z)
    p0, p1 = r["peaks"][0], r["peaks"][1]
    assert (int(p0["theta"]), int(p0["rho"]), int(p0["votes"])) == (ta, ba, int(keep_a.sum()))
    assert (int(p1["theta"]), int(p1["rho"]), int(p1["votes"])) == (tb, bb, int(keep_b.sum()))
    x = fp64_rho_bins(G, n_theta, n_rho, phi, z)
    checked = 0
    for h in range(len(phi)):
        da = abs(math.floor(x[h, ta]) - ba)
        db = abs(math.floor(x[h, tb]) - bb)
        eps = edge_margin(G, n_theta, n_rho)
        if not all(eps < fr < 1.0 - eps for fr in (x[h, ta] % 1.0, x[h, tb] % 1.0)):
            continue                         # FP64 and fixed point may differ by one bin here
        checked += 1
        if da <= 1:
            assert r["hit_track"][h] == 0
        elif db <= 1:
            assert r["hit_track"][h] == 1
        else:
            assert r["hit_track"][h] not in (0, 1)
    assert checked >= len(phi) - 3
    n_ab = int(keep_a.sum() + keep_b.sum())
    ht = r["hit_track"]
    assert ht[n_ab] == 0 and ht[n_ab + 2] == 0          # one bin off: on the line
    assert ht[n_ab + 1] != 0 and ht[n_ab + 3] != 0      # two bins off: not on it
    assert r["hit_track"][len(phi) - 1] == -1 or r["hit_track"][len(phi) - 1] >= 2


def test_rejected_hits_and_compaction_layout():
    """Hits outside the detector box (Section 2 ranges) are rejected (-2) and
    flagged; track_hits groups hits per peak in peak order, each group in
    increasing hit index, then the unassigned, then the rejected hits."""
    w = synth.generate(30, 5, (100.0, 300.0), 0.05, seed=2)
    phi, z = oracle.encode(G, w.vane, w.strip)
    phi[3] = 72000
    z[10] = -40000
    for k in range(w.n_windows):
        sl = w.window(k)
        r = oracle.find_window(G, 256, 256, phi[sl], z[sl])
        ht, th = r["hit_track"], r["track_hits"]
        n = sl.stop - sl.start
        assert sorted(th.tolist()) == list(range(n))
        pos = 0
        for p in range(r["n_peaks"]):
            pk = r["peaks"][p]
            assert pk["hit_begin"] == pos
            grp = th[pos:pos + pk["n_hits"]]
            assert np.all(np.diff(grp) > 0) and np.all(ht[grp] == p)
            pos += pk["n_hits"]
        rest = th[pos:]
        cats = ht[rest]
        assert np.all(np.diff(cats) <= 0)              # -1 block then -2 block
        for c in (-1, -2):
            grp = rest[cats == c]
            assert np.all(np.diff(grp) > 0)
        has_bad = np.any((phi[sl] == 72000) | (z[sl] == -40000))
        assert bool(r["status"] & oracle.WIN_HIT_OUT_OF_RANGE) == bool(has_bad)
        assert np.all((ht == -2) == ((phi[sl] == 72000) | (z[sl] == -40000)))


# --------------------------------------------------------------- invariants -

def test_permutation_invariance():
    """The window is a set of hits: reordering them leaves the accumulator and
    the peak list unchanged and permutes the assignment with them."""
    w = synth.generate(6, 8, (100.0, 300.0), 0.05, seed=4)
    phi, z = oracle.encode(G, w.vane, w.strip)
    rng = np.random.default_rng(0)
    for k in range(w.n_windows):
        sl = w.window(k)
        a = oracle.find_window(G, 512, 512, phi[sl], z[sl])
        perm = rng.permutation(sl.stop - sl.start)
        b = oracle.find_window(G, 512, 512, phi[sl][perm], z[sl][perm])
        np.testing.assert_array_equal(a["acc"], b["acc"])
        np.testing.assert_array_equal(a["peaks"][["theta", "rho", "votes", "n_hits"]],
                                      b["peaks"][["theta", "rho", "votes", "n_hits"]])
        np.testing.assert_array_equal(b["hit_track"], a["hit_track"][perm])


def test_truncation_keeps_the_best_and_flags_overflow():
    """The kept list is the head of the full sorted list; PEAK_OVERFLOW is set
    exactly when more peaks were found than kept."""
    w = synth.generate(4, 20, (100.0, 300.0), 0.05, seed=8)
    phi, z = oracle.encode(G, w.vane, w.strip)
    for k in range(w.n_windows):
        sl = w.window(k)
        full = oracle.find_window(G, 256, 256, phi[sl], z[sl], max_peaks=100000)
        for cap in (0, 1, 7, 64):
            r = oracle.find_window(G, 256, 256, phi[sl], z[sl], max_peaks=cap)
            assert r["n_found"] == full["n_found"]
            np.testing.assert_array_equal(r["peaks"][["theta", "rho", "votes"]],
                                          full["peaks"][:cap][["theta", "rho", "votes"]])
            assert bool(r["status"] & oracle.WIN_PEAK_OVERFLOW) == (full["n_found"] > cap)


def test_empty_and_small_windows():
    """No hits: empty accumulator, no peaks.  Fewer than T hits: no peak."""
    r = oracle.find_window(G, 64, 64, np.zeros(0, np.int32), np.zeros(0, np.int32))
    assert r["n_peaks"] == 0 and r["n_found"] == 0 and r["status"] == 0 and r["acc"].sum() == 0
    phi, z = _line_hits(100.5, 10.0, range(4))
    r = oracle.find_window(G, 64, 64, phi, z, vote_threshold=5)
    assert r["n_found"] == 0 and np.all(r["hit_track"] == -1)


def test_batch_equals_windows_one_by_one():
    w = synth.generate(12, ("poisson", 6, 1, 20), (100.0, 300.0), 0.02, seed=6)
    phi, z = oracle.encode(G, w.vane, w.strip)
    b = oracle.find_batch(G, 128, 256, phi, z, w.offsets, export_acc=True)
    for k in range(w.n_windows):
        sl = w.window(k)
        r = oracle.find_window(G, 128, 256, phi[sl], z[sl])
        np.testing.assert_array_equal(b["acc"][k], r["acc"])
        assert b["n_peaks"][k] == r["n_peaks"]
        np.testing.assert_array_equal(b["peaks"][k][: r["n_peaks"]], r["peaks"])
        np.testing.assert_array_equal(b["hit_track"][sl], r["hit_track"])
        np.testing.assert_array_equal(b["track_hits"][sl], r["track_hits"])
