"""Pins of the oracle's time slicing (Section 5: overlapping windows of 10 ns
sliding by 5 ns) against a hand-worked example and closed forms."""
import os

import numpy as np
import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))


def _read_example():
    d, wins = {}, {}
    for ln in open(os.path.join(HERE, "golden", "time_slice_example.txt")):
        ln = ln.split("#")[0].split()
        if not ln:
            continue
        if ln[0].startswith("w") and ln[0][1:].isdigit():
            wins[int(ln[0][1:])] = [int(x) for x in ln[1:]]
        else:
            d[ln[0]] = [int(x) for x in ln[1:]]
    return d, wins


def test_hand_worked_example():
    d, wins = _read_example()
    offs, idx = oracle.time_slice(np.array(d["t"]), d["t0"][0], d["step"][0], d["len"][0],
                                  d["windows"][0])
    for k in range(d["windows"][0]):
        assert list(idx[offs[k]:offs[k + 1]]) == wins[k], k


@pytest.mark.parametrize("m", [1, 2, 3])
def test_membership_closed_form(m):
    """Every hit appears in exactly the windows k with
    floor((t - t0 - len)/step) < k <= floor((t - t0)/step), 0 <= k < W."""
    rng = np.random.default_rng(m)
    step, t0, W = 5000, -2500, 300
    t = np.sort(rng.integers(-20000, 1_560_000, 4000))
    offs, idx = oracle.time_slice(t, t0, step, m * step, W)
    hi = np.floor_divide(t - t0, step)
    lo = np.floor_divide(t - t0 - m * step, step)
    expect = np.clip(np.minimum(hi, W - 1) - np.maximum(lo, -1), 0, None)
    got = np.bincount(idx, minlength=len(t))
    np.testing.assert_array_equal(got, expect)
    # each window is a contiguous, increasing run of the sorted input
    for k in range(W):
        run = idx[offs[k]:offs[k + 1]]
        if len(run):
            np.testing.assert_array_equal(run, np.arange(run[0], run[0] + len(run)))
            assert (t[run] >= t0 + k * step).all() and (t[run] < t0 + k * step + m * step).all()


def test_one_step_windows_partition_the_covered_span():
    rng = np.random.default_rng(7)
    t = np.sort(rng.integers(0, 100_000, 2000))
    offs, idx = oracle.time_slice(t, 10_000, 1000, 1000, 50)
    inside = np.nonzero((t >= 10_000) & (t < 60_000))[0]
    np.testing.assert_array_equal(np.sort(idx), inside)
    assert len(np.unique(idx)) == len(idx)


def test_input_order_is_kept_for_unsorted_times():
    """The definition does not need sorted times: a window lists its hits in
    input order, so a permuted input gives the permuted lists."""
    rng = np.random.default_rng(3)
    t = rng.integers(0, 50_000, 500)
    perm = rng.permutation(len(t))
    o1, i1 = oracle.time_slice(t, 0, 5000, 10000, 10)
    o2, i2 = oracle.time_slice(t[perm], 0, 5000, 10000, 10)
    np.testing.assert_array_equal(o1, o2)
    for k in range(10):
        a = set(i1[o1[k]:o1[k + 1]].tolist())
        b = i2[o2[k]:o2[k + 1]]
        assert set(perm[b].tolist()) == a
        assert (np.diff(b) > 0).all()


def test_empty_and_out_of_range():
    offs, idx = oracle.time_slice(np.zeros(0, np.int64), 0, 5, 10, 4)
    assert list(offs) == [0] * 5 and len(idx) == 0
    offs, idx = oracle.time_slice(np.array([-1, 100]), 0, 5, 10, 4)
    assert len(idx) == 0
