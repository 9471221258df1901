"""Pins of the oracle's track extension (Section 4: a seed of three hits on
consecutive vanes, extrapolated to neighbouring vanes) and of the efficiency
of Section 7 (found = hits on five continuous vanes).

The extension pins are hand-built windows whose answer follows in closed
form: collinear and parabolic tracks (where the three-point extrapolation is
exact), the tolerance edge, the tie rules, claiming by an earlier track, the
ring of vanes and the seed choice.  Coordinates are written out from the
detector's units: phi = 9 deg * vane at 200 units per degree, z = the centre
of the strip, 38 units per 0.19 mm strip from z_min = -38912.
"""
import numpy as np
import pytest

import oracle
from paper_2511_02742_gb300 import evaluate, synth

G = synth.GEOMETRY
PITCH = 38
TOL = 16 * PITCH


def enc(vanes, strips):
    v = np.asarray(vanes, np.int64)
    s = np.asarray(strips, np.int64)
    return (1800 * v).astype(np.int32), (-38912 + PITCH * s + PITCH // 2).astype(np.int32)


def run(vanes, strips, groups, tol=TOL, rejected=()):
    phi, z = enc(vanes, strips)
    return oracle.extend_window(G, phi, z, groups, tol, rejected=rejected)


def by_vane(idx, vanes):
    return list(np.asarray(idx)[np.argsort(np.asarray(vanes)[idx], kind="stable")])


def test_collinear_track_is_extended_from_its_seed_both_ways():
    rng = np.random.default_rng(1)
    vanes = list(range(5, 15))
    strips = [100 + 7 * (v - 5) for v in vanes]
    # distractors just outside the tolerance on every vane
    for v in range(5, 15):
        vanes += [v, v]
        strips += [100 + 7 * (v - 5) + 17, 100 + 7 * (v - 5) - 17]
    perm = rng.permutation(len(vanes))
    vanes = np.asarray(vanes)[perm]
    strips = np.asarray(strips)[perm]
    true_idx = [int(np.flatnonzero((vanes == v) & (strips == 100 + 7 * (v - 5)))[0])
                for v in range(5, 15)]
    seed = sorted(true_idx[4:7])                       # the hits on vanes 9, 10, 11
    ext, ext_track, ext_hits = run(vanes, strips, [seed])
    assert ext[0]["n_hits"] == 10 and ext[0]["first_vane"] == 5 and ext[0]["hit_begin"] == 0
    assert ext[0]["seed_mid"] == true_idx[5]
    assert list(ext_hits[:10]) == true_idx              # increasing vane order
    assert sorted(np.flatnonzero(ext_track == 0)) == sorted(true_idx)
    assert sorted(ext_hits[10:]) == sorted(set(range(len(vanes))) - set(true_idx))
    assert list(ext_hits[10:]) == sorted(ext_hits[10:])


def test_parabolic_track_is_followed_exactly():
    """z = a + b k + c k^2 in strips: the parabola through the last three hits
    predicts the next one exactly, so a distractor one strip off never wins."""
    ks = np.arange(13)
    strips = 500 + 3 * ks + 2 * ks * ks
    vanes = list(ks) + list(ks[3:])
    all_strips = list(strips) + list(strips[3:] - 1)
    ext, ext_track, ext_hits = run(vanes, all_strips, [[0, 1, 2]])
    assert ext[0]["n_hits"] == 13 and ext[0]["first_vane"] == 0
    assert list(ext_hits[:13]) == list(range(13))
    assert (ext_track[13:] == -1).all()


def test_tolerance_edge_is_inclusive():
    # flat seed on vanes 0-2; vane 3 offers z exactly pred + tol; vane 4 offers
    # pred + tol + 1 strip, where pred = 3*1016 - 3*1000 + 1000 = 1048 strips
    vanes = [0, 1, 2, 3, 4]
    strips = [1000, 1000, 1000, 1016, 1048 + 17]
    ext, ext_track, _ = run(vanes, strips, [[0, 1, 2]])
    assert ext[0]["n_hits"] == 4 and ext[0]["first_vane"] == 0
    assert list(ext_track) == [0, 0, 0, 0, -1]
    # one z unit beyond the tolerance is out
    ext, ext_track, _ = run(vanes[:4], strips[:4], [[0, 1, 2]], tol=TOL - 1)
    assert ext[0]["n_hits"] == 3 and ext_track[3] == -1


def test_ties_take_the_lower_z_then_the_lower_index():
    # vane 3: 995 and 1005 are equally near 1000 -> 995; then the prediction on
    # vane 4 is 3*995 - 3*1000 + 1000 = 985, offered twice -> the lower index
    vanes = [0, 1, 2, 3, 3, 4, 4]
    strips = [1000, 1000, 1000, 1005, 995, 985, 985]
    ext, ext_track, ext_hits = run(vanes, strips, [[0, 1, 2]])
    assert ext[0]["n_hits"] == 5
    assert list(ext_hits[:5]) == [0, 1, 2, 4, 5]
    assert list(ext_track) == [0, 0, 0, -1, 0, 0, -1]


def test_claimed_hits_are_not_reused():
    vanes = list(range(10, 18))
    strips = [300] * 8
    groups = [[0, 1, 2], [4, 5, 6], []]
    ext, ext_track, ext_hits = run(vanes, strips, groups)
    assert ext[0]["n_hits"] == 8
    for p in (1, 2):       # everything was taken by the first track; an empty group
        assert ext[p]["n_hits"] == 0 and ext[p]["first_vane"] == -1
        assert ext[p]["seed_mid"] == -1 and ext[p]["hit_begin"] == 8
    assert (ext_track == 0).all()


def test_second_track_keeps_its_own_hits():
    # two parallel lines 40 strips apart: each seed extends along its own line
    vanes = list(range(0, 8)) * 2
    strips = [200 + 4 * v for v in range(8)] + [240 + 4 * v for v in range(8)]
    ext, ext_track, ext_hits = run(vanes, strips, [[8, 9, 10], [3, 4, 5]])
    assert ext[0]["n_hits"] == 8 and ext[1]["n_hits"] == 8
    assert list(ext_hits[:8]) == list(range(8, 16))
    assert list(ext_hits[8:16]) == list(range(8))
    assert ext[1]["hit_begin"] == 8


@pytest.mark.parametrize("seed", [[1, 2, 3], [0, 1, 2], [4, 5, 6]])
def test_extension_wraps_around_the_ring_of_vanes(seed):
    """A line over vanes 37..39, 0..3: seeded across the joint, before it
    (forward crosses 39 -> 0) and after it (backward crosses 0 -> 39)."""
    vanes = [37, 38, 39, 0, 1, 2, 3]
    strips = [200 + 5 * k for k in range(7)]
    ext, ext_track, ext_hits = run(vanes, strips, [seed])
    assert ext[0]["n_hits"] == 7 and ext[0]["first_vane"] == 37
    assert list(ext_hits) == list(range(7))


def test_a_track_never_exceeds_the_number_of_vanes():
    """A flat line on all 40 vanes plus a second hit on vane 39: the seed with
    the lowest middle index is (39, 0, 1); forward reaches vane 38, the ring is
    full and the second hit on vane 39 stays free."""
    vanes = list(range(40)) + [39]
    strips = [700] * 41
    ext, ext_track, ext_hits = run(vanes, strips, [list(range(40))])
    assert ext[0]["n_hits"] == 40 and ext[0]["first_vane"] == 39 and ext[0]["seed_mid"] == 0
    assert list(ext_hits) == [39] + list(range(39)) + [40]
    assert ext_track[40] == -1


def test_seed_is_the_straightest_triplet_then_the_lowest_indices():
    # triplet on vanes 3-5 bends by 2 strips, the one on 20-22 is straight
    vanes = [3, 4, 5, 20, 21, 22]
    strips = [100, 100, 102, 900, 905, 910]
    ext, _, _ = run(vanes, strips, [list(range(6))], tol=TOL)
    assert ext[0]["seed_mid"] == 4
    # equal bends: the lower middle index wins
    vanes = [20, 21, 22, 3, 4, 5]
    strips = [900, 905, 910, 100, 100, 100]
    ext, _, _ = run(vanes, strips, [list(range(6))])
    assert ext[0]["seed_mid"] == 1


def test_seed_bend_is_bounded_by_the_tolerance():
    ext, _, _ = run([0, 1, 2], [1000, 1000, 1017], [[0, 1, 2]])
    assert ext[0]["n_hits"] == 0 and ext[0]["seed_mid"] == -1
    ext, _, _ = run([0, 1, 2], [1000, 1000, 1016], [[0, 1, 2]])
    assert ext[0]["n_hits"] == 3


def test_rejected_and_off_vane_hits_take_no_part():
    vanes = [0, 1, 2, 3, 4]
    strips = [500] * 5
    phi, z = enc(vanes, strips)
    phi[4] += 1                      # not on a vane
    ext, ext_track, _ = oracle.extend_window(G, phi, z, [[0, 1, 2]], TOL, rejected=[3])
    assert ext[0]["n_hits"] == 3 and list(ext_track) == [0, 0, 0, -1, -1]


def test_invariants_on_generated_windows():
    """On pileup windows through the oracle's steps A-D: ext_hits is a
    permutation per window; each track sits on consecutive vanes from its first
    vane, one hit per vane; every hit beyond the seed is within the tolerance
    of the three-point prediction from its neighbours towards the seed."""
    w = synth.generate(40, ("poisson", 8, 1, 20), (100.0, 300.0), 0.02, seed=12)
    phi, z = oracle.encode(G, w.vane, w.strip)
    f = oracle.find_batch(G, 180, 256, phi, z, w.offsets)
    ext, ext_track, ext_hits = oracle.extend(G, phi, z, w.offsets, f, TOL)
    n_tracks = 0
    for win in range(w.n_windows):
        s = w.window(win)
        n = s.stop - s.start
        assert sorted(ext_hits[s]) == list(range(n))
        v = w.vane[s]
        zz = z[s].astype(np.int64)
        for p in range(f["n_peaks"][win]):
            e = ext[win, p]
            mine = np.flatnonzero(ext_track[s] == p)
            assert len(mine) == e["n_hits"]
            if e["n_hits"] == 0:
                continue
            n_tracks += 1
            hs = ext_hits[s][e["hit_begin"]: e["hit_begin"] + e["n_hits"]]
            assert sorted(hs) == sorted(mine)
            assert list(v[hs]) == [(e["first_vane"] + k) % 40 for k in range(e["n_hits"])]
            m = list(hs).index(e["seed_mid"])
            for k in range(len(hs)):
                if k >= m + 2:
                    pred = 3 * zz[hs[k - 1]] - 3 * zz[hs[k - 2]] + zz[hs[k - 3]]
                elif k <= m - 2:
                    pred = 3 * zz[hs[k + 1]] - 3 * zz[hs[k + 2]] + zz[hs[k + 3]]
                else:
                    continue
                assert abs(zz[hs[k]] - pred) <= TOL
    assert n_tracks > 100


def test_clean_high_momentum_tracks_are_found():
    """Section 7: tracks above 200 MeV/c leave enough hits; one clean track per
    window is found (hits on five continuous vanes in one extended track)."""
    w = synth.generate(200, 1, (200.0, 300.0), 0.0, seed=5)
    phi, z = oracle.encode(G, w.vane, w.strip)
    f = oracle.find_batch(G, 512, 512, phi, z, w.offsets)
    _, ext_track, _ = oracle.extend(G, phi, z, w.offsets, f, TOL)
    e = evaluate.efficiency(w.vane, w.track, w.offsets, w.track_offsets, ext_track)
    assert e["findable"] >= 150
    assert e["epsilon_findable"] >= 0.9


# ------------------------------------------------------------ efficiency pins

@pytest.mark.parametrize("vanes, ext, found, findable", [
    ([3, 4, 5, 6, 7], [0] * 5, 1, 1),                   # five continuous vanes
    ([3, 4, 5, 7, 8], [0] * 5, 0, 0),                   # a gap: not even findable
    ([38, 39, 0, 1, 2], [0] * 5, 1, 1),                 # across the ring's joint
    ([3, 4, 5, 6, 7], [0, 0, 0, 1, 1], 0, 1),           # split between two tracks
    ([3, 4, 5, 6, 7], [0, 0, -1, 0, 0], 0, 1),          # a hit not taken
    ([3, 4, 5, 6, 7, 8], [1, 0, 0, 0, 0, 0], 1, 1),     # five of six in one track
    (list(range(40)), [0] * 40, 1, 1),                  # the whole ring
])
def test_efficiency_definition(vanes, ext, found, findable):
    n = len(vanes)
    e = evaluate.efficiency(np.array(vanes), np.zeros(n, np.int32), np.array([0, n]),
                            np.array([0, 1]), np.array(ext))
    assert e["found"] == found and e["all"] == 1 and e["findable"] == findable


def test_efficiency_counts_every_generated_track():
    # window 0: track 0 found, track 1 has only three hits; window 1: noise only
    vanes = np.array([0, 1, 2, 3, 4, 10, 11, 12, 20, 21])
    truth = np.array([0, 0, 0, 0, 0, 1, 1, 1, -1, -1])
    ext = np.array([2, 2, 2, 2, 2, 0, 0, 0, -1, -1])
    e = evaluate.efficiency(vanes, truth, np.array([0, 8, 10]), np.array([0, 2, 2]), ext)
    assert e == dict(found=1, all=2, epsilon=0.5, findable=1, epsilon_findable=1.0)
