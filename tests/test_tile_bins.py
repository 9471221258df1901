"""The find's narrowed tiles (hough_tile_bins, host only, no GPU): every bin
that a hit of the detector box can vote in a tile's rows lies in the tile's
stored bins [lo, lo + NB), NB and lo follow the documented rule, and the
layout leaves nothing reachable out.  The reachable bins come from the
oracle's own fixed-point bins (`oracle.bins_fixed`) of the box's corners
(the bin is monotone in phi and in z) and of random hits of the box."""
import numpy as np
import pytest

import oracle
from paper_2511_02742_gb300 import synth

G = synth.GEOMETRY
PHI_END = 360 * G["phi_u_per_deg"]                      # phi in [0, PHI_END)
Z_LO = G["z_min_u"]
Z_HI = G["z_min_u"] + G["n_z_strips"] * G["z_pitch_u"]   # z in [Z_LO, Z_HI]
CORNERS = ([0, 0, PHI_END - 1, PHI_END - 1], [Z_LO, Z_HI, Z_LO, Z_HI])
SHAPES = [(512, 512), (1024, 1024), (180, 1000), (97, 332), (256, 256), (33, 64), (128, 512),
          (1, 4)]


@pytest.fixture(scope="module")
def hough():
    from paper_2511_02742_gb300 import build, hough
    build.build()
    return hough


def row_reach(n_theta, n_rho):
    """Lowest and highest bin per row over the box (the corners bound it)."""
    b = oracle.bins_fixed(G, n_theta, n_rho, *CORNERS)      # [4, n_theta]
    return b.min(axis=0), b.max(axis=0)


def tiles(n_theta, word_rows, k):
    r = word_rows << k
    return [(i, i * r, min(n_theta, (i + 1) * r)) for i in range((n_theta + r - 1) // r)]


@pytest.mark.parametrize("n_theta,n_rho", SHAPES)
@pytest.mark.parametrize("word_rows", [32, 64, 128])
def test_layout_rule_and_cover(hough, n_theta, n_rho, word_rows):
    nb, lo = hough.hough_tile_bins(G, n_theta, n_rho, word_rows)
    assert lo.shape == (3, (n_theta + 31) // 32)
    assert nb % 4 == 0 and 4 <= nb <= n_rho
    rlo, rhi = row_reach(n_theta, n_rho)
    widest = 1
    for k in range(3):
        ts = tiles(n_theta, word_rows, k)
        assert (lo[k, len(ts):] == 0).all()
        for i, a, b in ts:
            low, high = int(rlo[a:b].min()), int(rhi[a:b].max())
            first, last = max(low, 0), min(high, n_rho - 1)
            if last >= first:
                widest = max(widest, last - first + 1)
            l0 = int(lo[k, i])
            assert l0 % 4 == 0 and 0 <= l0 <= n_rho - nb, (k, i, l0)
            if last >= first:
                # every reachable bin inside [0, n_rho) is stored
                assert l0 <= first and last < l0 + nb, (k, i, l0, first, last)
            if low < 0:
                assert l0 == 0
    assert nb == min((widest + 3 + 3) // 4 * 4, n_rho)


@pytest.mark.parametrize("n_theta,n_rho", [(512, 512), (180, 1000), (97, 332)])
def test_random_box_hits_vote_inside_the_stored_bins(hough, n_theta, n_rho):
    rng = np.random.default_rng(5)
    phi = np.r_[rng.integers(0, PHI_END, 4000), CORNERS[0]].astype(np.int32)
    z = np.r_[rng.integers(Z_LO, Z_HI + 1, 4000), CORNERS[1]].astype(np.int32)
    bins = oracle.bins_fixed(G, n_theta, n_rho, phi, z)      # [H, n_theta]
    for word_rows in (32, 64):
        nb, lo = hough.hough_tile_bins(G, n_theta, n_rho, word_rows)
        for k in range(3):
            for i, a, b in tiles(n_theta, word_rows, k):
                v = bins[:, a:b]
                v = v[(v >= 0) & (v < n_rho)]
                assert ((v >= lo[k, i]) & (v < lo[k, i] + nb)).all(), (word_rows, k, i)


def test_full_width_where_nothing_can_be_left_out(hough):
    """With one 4-bin accumulator row the tile stores every bin from 0."""
    nb, lo = hough.hough_tile_bins(G, 1, 4, 32)
    assert nb == 4 and (lo == 0).all()


def test_invalid_arguments(hough):
    with pytest.raises(hough.HoughError):
        hough.hough_tile_bins(G, 512, 512, 48)
    with pytest.raises(hough.HoughError):
        hough.hough_tile_bins(G, 512, 510, 32)
