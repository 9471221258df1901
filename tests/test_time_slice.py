"""Device time slicing (hough_time_slice) against the oracle's definition,
and the whole chain -- slice, then vote/peaks/association -- against the
oracle's slice followed by the oracle's find."""
import numpy as np
import pytest

import oracle
from paper_2511_02742_gb300 import synth

pytestmark = pytest.mark.gpu
G = synth.GEOMETRY


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _slice(f, s, t0, step, length, W):
    import torch
    r = f.time_slice(_dev(s.t), dict(vane=_dev(s.vane), strip=_dev(s.strip)), t0, step, length, W)
    torch.cuda.synchronize()
    return r


@pytest.mark.parametrize("m,t0", [(2, 0), (1, -3000), (4, 1234)])
def test_slice_matches_oracle(hough, m, t0):
    s = synth.timed_stream(4000, 0.6, noise_frac=0.02, seed=m)      # 4 us, ~3.4e4 hits
    step = 5000                                                      # 5 ns in ps
    W = int(4000 * 1000 // step) + 2
    f = hough.Finder(512, 512)
    r = _slice(f, s, t0, step, m * step, W)
    offs, idx = oracle.time_slice(s.t, t0, step, m * step, W)
    np.testing.assert_array_equal(r["offsets"].cpu().numpy(), offs)
    n = len(idx)
    np.testing.assert_array_equal(r["index"].cpu().numpy()[:n], idx)
    np.testing.assert_array_equal(r["hits"]["vane"].cpu().numpy()[:n], s.vane[idx])
    np.testing.assert_array_equal(r["hits"]["strip"].cpu().numpy()[:n], s.strip[idx])
    assert int(r["status"].item()) == 0
    f.close()


def test_slice_then_find_matches_oracle_chain(hough):
    import torch
    s = synth.timed_stream(3000, 0.6, noise_frac=0.02, seed=11)
    step, W = 5000, 601
    f = hough.Finder(512, 512)
    r = _slice(f, s, 0, step, 2 * step, W)
    out = f.alloc_outputs(W, r["capacity"])
    f.find(r["hits"], r["offsets"], out=out)
    torch.cuda.synchronize()
    offs, idx = oracle.time_slice(s.t, 0, step, 2 * step, W)
    phi, z = oracle.encode(G, s.vane[idx], s.strip[idx])
    ref = oracle.find_batch(G, 512, 512, phi, z, offs)
    n = len(idx)
    np.testing.assert_array_equal(out["n_peaks"].cpu().numpy(), ref["n_peaks"])
    np.testing.assert_array_equal(out["n_found"].cpu().numpy(), ref["n_found"])
    np.testing.assert_array_equal(out["hit_track"].cpu().numpy()[:n], ref["hit_track"])
    np.testing.assert_array_equal(out["track_hits"].cpu().numpy()[:n], ref["track_hits"])
    pk = hough.decode_peaks(out["peaks"])
    for k in range(W):
        c = int(ref["n_peaks"][k])
        np.testing.assert_array_equal(pk[k][:c], ref["peaks"][k][:c])
    assert (np.diff(offs) > 0).sum() > W // 2
    f.close()


def test_edges_empty_stream_and_unsorted(hough):
    import torch
    f = hough.Finder(256, 256)
    # hits before t0 and past the last window are left out; empty windows
    t = np.array([-5, 0, 1, 40, 41, 42, 500, 10_000], np.int64)
    vane = np.arange(8, dtype=np.int32)
    strip = np.arange(8, dtype=np.int32) * 3
    s = synth.TimedHits(t, vane, strip, np.zeros(8, np.int64))
    r = _slice(f, s, 0, 10, 20, 30)
    offs, idx = oracle.time_slice(t, 0, 10, 20, 30)
    np.testing.assert_array_equal(r["offsets"].cpu().numpy(), offs)
    np.testing.assert_array_equal(r["index"].cpu().numpy()[:len(idx)], idx)
    # an empty stream: every window empty
    e = synth.TimedHits(np.zeros(0, np.int64), np.zeros(0, np.int32), np.zeros(0, np.int32),
                        np.zeros(0, np.int64))
    r = _slice(f, e, 0, 10, 20, 7)
    assert r["offsets"].cpu().numpy().tolist() == [0] * 8
    # unsorted times are reported, and nothing outside the arrays is written
    u = synth.TimedHits(t[::-1].copy(), vane, strip, np.zeros(8, np.int64))
    r = _slice(f, u, 0, 10, 20, 30)
    assert int(r["status"].item()) == hough.HOUGH_SLICE_UNSORTED
    # a window length that is not a whole number of steps is refused
    with pytest.raises(hough.HoughError) as ex:
        f.time_slice(_dev(t), dict(vane=_dev(vane), strip=_dev(strip)), 0, 10, 25, 4)
    assert ex.value.code == hough.HOUGH_ERR_UNSUPPORTED_SHAPE
    f.close()


@pytest.mark.parametrize("rate,m,W", [(0.002, 2, 257), (0.6, 16, 1500), (0.05, 3, 256),
                                      (0.6, 1, 1), (0.3, 7, 2049)])
def test_blocks_gaps_and_duplicate_times(hough, rate, m, W):
    """Window counts around the slicer's block of 256 windows, sparse streams
    (many window starts between two hits), the longest overlap, and repeated
    times (a lower bound takes the first of equal times)."""
    step = 5000
    s = synth.timed_stream(W * step / 1000.0 + 50, rate, noise_frac=0.02, seed=W)
    t = s.t.copy()
    t[1::7] = t[0::7][:len(t[1::7])]            # repeat some times (still sorted)
    t = np.maximum.accumulate(t)
    f = hough.Finder(256, 256)
    r = _slice(f, synth.TimedHits(t, s.vane, s.strip, s.track), -777, step, m * step, W)
    offs, idx = oracle.time_slice(t, -777, step, m * step, W)
    np.testing.assert_array_equal(r["offsets"].cpu().numpy(), offs)
    np.testing.assert_array_equal(r["index"].cpu().numpy()[:len(idx)], idx)
    assert int(r["status"].item()) == 0
    f.close()


def test_extreme_times(hough):
    """Times near the ends of int64 lie before or after every window."""
    big = np.iinfo(np.int64)
    t = np.array([big.min, big.min + 5, -20, 0, 3, 3, 17, 29, big.max - 9, big.max], np.int64)
    vane = np.arange(len(t), dtype=np.int32)
    f = hough.Finder(256, 256)
    r = _slice(f, synth.TimedHits(t, vane, vane, np.zeros(len(t), np.int64)), 0, 10, 20, 5)
    offs, idx = oracle.time_slice(t, 0, 10, 20, 5)
    np.testing.assert_array_equal(r["offsets"].cpu().numpy(), offs)
    np.testing.assert_array_equal(r["index"].cpu().numpy()[:len(idx)], idx)
    f.close()
