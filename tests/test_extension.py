"""The track-extension kernel (hough_extend) against the oracle, bit-exact:
every peak's extended track (first vane, hit count, place in ext_hits, seed),
every hit's track and the per-window hit order.  Each side runs on its own
step A-D output (the GPU's from hough_find, the oracle's from its own find),
which are themselves bit-exact."""
import numpy as np
import pytest

import oracle
from paper_2511_02742_gb300 import evaluate, synth

pytestmark = pytest.mark.gpu
G = synth.GEOMETRY
TOL = 16 * 38


def _gpu(hough, w, n_theta, n_rho, tol, raw=True, phi=None, z=None, max_peaks=64):
    import torch
    f = hough.Finder(n_theta, n_rho, max_peaks=max_peaks)
    if raw:
        hits = dict(vane=torch.from_numpy(w.vane).cuda(), strip=torch.from_numpy(w.strip).cuda())
    else:
        hits = dict(phi_q=torch.from_numpy(phi).cuda(), z_q=torch.from_numpy(z).cuda())
    offs = torch.from_numpy(w.offsets).cuda()
    found = f.find(hits, offs)
    nh = max(w.n_hits, 1)
    out = dict(tracks=torch.full((w.n_windows, max_peaks, 4), -7, dtype=torch.int32, device="cuda"),
               ext_track=torch.full((nh,), -7, dtype=torch.int32, device="cuda"),
               ext_hits=torch.full((nh,), -7, dtype=torch.int32, device="cuda"),
               window_status=torch.full((max(w.n_windows, 1),), -7, dtype=torch.int32,
                                        device="cuda"))
    f.extend(hits, offs, found, tol, out=out)
    torch.cuda.synchronize()
    n_peaks = found["n_peaks"].cpu().numpy()
    launches = f.launch_count() if hasattr(f, "launch_count") else None
    f.close()
    return (out["tracks"].cpu().numpy().view(hough.EXT_DTYPE).reshape(w.n_windows, max_peaks),
            out["ext_track"].cpu().numpy()[:w.n_hits], out["ext_hits"].cpu().numpy()[:w.n_hits],
            out["window_status"].cpu().numpy()[:w.n_windows], n_peaks, launches)


def _oracle(w, n_theta, n_rho, tol, phi=None, z=None, max_peaks=64):
    if phi is None:
        phi, z = oracle.encode(G, w.vane, w.strip)
    f = oracle.find_batch(G, n_theta, n_rho, phi, z, w.offsets, max_peaks=max_peaks)
    ext, et, eh = oracle.extend(G, phi, z, w.offsets, f, tol)
    return ext, et, eh, f["n_peaks"]


def _check(hough, w, n_theta, n_rho, tol=TOL, raw=True, phi=None, z=None, max_peaks=64):
    ge, gt, gh, gs, gnp, _ = _gpu(hough, w, n_theta, n_rho, tol, raw, phi, z, max_peaks)
    re, rt, rh, rnp = _oracle(w, n_theta, n_rho, tol, phi, z, max_peaks)
    np.testing.assert_array_equal(gnp, rnp)
    for k in range(w.n_windows):
        np.testing.assert_array_equal(ge[k][:gnp[k]], re[k][:rnp[k]], err_msg=f"window {k}")
    np.testing.assert_array_equal(gt, rt)
    np.testing.assert_array_equal(gh, rh)
    assert (gs == 0).all()
    return ge, gt, gnp


@pytest.mark.parametrize("raw", [True, False])
def test_tiny_and_plain(hough, raw):
    for name in ("tiny", "plain"):
        w = synth.workload(name, n_windows=None if name == "tiny" else 80, seed=51)
        nt, nr = (256, 256) if name == "tiny" else (512, 512)
        phi, z = oracle.encode(G, w.vane, w.strip)
        ext, _, n_peaks = _check(hough, w, nt, nr, raw=raw, phi=phi, z=z)
        assert sum((ext[k][:n_peaks[k]]["n_hits"] > 0).sum() for k in range(w.n_windows)) > 0


def test_uneven_windows_with_empty_ones(hough):
    w = synth.concat([synth.generate(150, ("poisson", 10, 0, 40), (100.0, 300.0), 0.02, seed=52),
                      synth.generate(5, 0, (100.0, 300.0), 0.02, seed=59),
                      synth.generate(150, ("poisson", 3, 0, 40), (100.0, 300.0), 0.02, seed=60)])
    assert (np.diff(w.offsets) == 0).sum() >= 5
    _check(hough, w, 512, 512)


def test_windows_of_every_launch_tier(hough):
    """Windows up to 512 hits go to the first launch, up to 1536 to the
    second, up to 4096 to the third: all three kinds are present, interleaved,
    and all are exact."""
    w = synth.concat([synth.workload("high_pileup", n_windows=12, seed=53),
                      synth.generate(6, ("poisson", 10, 1, 40), (100.0, 300.0), 0.02, seed=61),
                      synth.generate(2, 110, (100.0, 300.0), 0.05, seed=62)])
    w = w.subset(np.random.default_rng(63).permutation(w.n_windows))
    n = np.diff(w.offsets)
    assert (n <= 512).any() and ((n > 512) & (n <= 1536)).any(), n
    assert ((n > 1536) & (n <= 4096)).any(), n
    _check(hough, w, 1024, 1024, max_peaks=256)


@pytest.mark.parametrize("tol", [0, 38, 3 * 38, (1 << 19) - 1])
def test_tolerance_range(hough, tol):
    w = synth.generate(120, ("poisson", 8, 1, 30), (100.0, 300.0), 0.05, seed=54)
    _check(hough, w, 512, 512, tol=tol)


def test_off_vane_and_out_of_box_hits(hough):
    """Encoded hits off the vane angles take no part; hits outside the box are
    rejected by the find step and take no part either."""
    w = synth.generate(100, ("poisson", 8, 1, 30), (100.0, 300.0), 0.02, seed=55)
    phi, z = oracle.encode(G, w.vane, w.strip)
    rng = np.random.default_rng(55)
    k = rng.choice(w.n_hits, w.n_hits // 20, replace=False)
    phi[k] += rng.integers(1, 1799, len(k)).astype(np.int32)
    k2 = rng.choice(w.n_hits, w.n_hits // 50, replace=False)
    z[k2] = 99999
    _check(hough, w, 512, 512, raw=False, phi=phi, z=z)


def test_oversized_window_is_flagged(hough):
    """A window of more than HOUGH_EXT_MAX_HITS hits gets no track and the
    TOO_LARGE status; its neighbours are extended as usual."""
    big = synth.generate(1, 200, (100.0, 300.0), 0.5, seed=56)
    assert big.n_hits > hough.HOUGH_EXT_MAX_HITS
    small = synth.generate(3, 5, (100.0, 300.0), 0.01, seed=57)
    w = synth.concat([small.subset([0]), big, small.subset([1, 2])])
    ge, gt, gh, gs, gnp, _ = _gpu(hough, w, 512, 512, TOL)
    assert list(gs) == [0, hough.HOUGH_WIN_TOO_LARGE, 0, 0]
    s = w.window(1)
    assert (gt[s] == -1).all() and (gh[s] == np.arange(s.stop - s.start)).all()
    assert (ge[1][:gnp[1]]["n_hits"] == 0).all() and (ge[1][:gnp[1]]["first_vane"] == -1).all()
    re, rt, rh, rnp = _oracle(w.subset([0, 2, 3]), 512, 512, TOL)
    for j, k in enumerate([0, 2, 3]):
        np.testing.assert_array_equal(ge[k][:gnp[k]], re[j][:rnp[j]])
        sk = w.window(k)
        sj = slice(int(w.subset([0, 2, 3]).offsets[j]), int(w.subset([0, 2, 3]).offsets[j + 1]))
        np.testing.assert_array_equal(gt[sk], rt[sj])
        np.testing.assert_array_equal(gh[sk], rh[sj])


def test_bad_arguments_are_rejected(hough):
    import torch
    f = hough.Finder(64, 64)
    w = synth.workload("tiny")
    hits = dict(vane=torch.from_numpy(w.vane).cuda(), strip=torch.from_numpy(w.strip).cuda())
    offs = torch.from_numpy(w.offsets).cuda()
    found = f.find(hits, offs)
    for tol in (-1, hough.HOUGH_EXT_MAX_TOL + 1):
        with pytest.raises(hough.HoughError) as e:
            f.extend(hits, offs, found, tol)
        assert e.value.code == -1
    f.close()


def test_efficiency_is_the_same_from_either_side(hough):
    """Section 7's efficiency computed from the GPU's ext_track equals the one
    from the oracle's (a consequence of bit-exactness, checked end to end)."""
    w = synth.generate(400, ("poisson", 10, 1, 40), (100.0, 300.0), 0.02, seed=58)
    _, gt, _, _, _, _ = _gpu(hough, w, 512, 512, TOL)
    _, rt, _, _ = _oracle(w, 512, 512, TOL)
    a = evaluate.efficiency(w.vane, w.track, w.offsets, w.track_offsets, gt)
    b = evaluate.efficiency(w.vane, w.track, w.offsets, w.track_offsets, rt)
    assert a == b and a["epsilon_findable"] > 0.6


def test_bad_offsets_are_flagged_not_read(hough):
    """Windows whose offsets run backwards or past the hits get
    HOUGH_WIN_BAD_OFFSETS; the valid windows around them are exact."""
    import torch
    w = synth.generate(6, 5, (100.0, 300.0), 0.01, seed=64)
    f = hough.Finder(512, 512)
    hits = dict(vane=torch.from_numpy(w.vane).cuda(), strip=torch.from_numpy(w.strip).cuda())
    good = torch.from_numpy(w.offsets).cuda()
    found = f.find(hits, good)
    bad = w.offsets.copy()
    bad = np.concatenate([bad, [bad[-1] + 1000, bad[2]]])      # past n_hits, then backwards
    offs = torch.from_numpy(bad).cuda()
    nw = len(bad) - 1
    fb = f.alloc_outputs(nw, w.n_hits)
    f.find(hits, offs, out=fb)
    ext = f.extend(hits, offs, fb, TOL)
    ref = f.extend(hits, good, found, TOL)
    torch.cuda.synchronize()
    st = ext["window_status"].cpu().numpy()[:nw]
    assert list(st[w.n_windows:]) == [hough.HOUGH_WIN_BAD_OFFSETS] * 2
    assert (st[:w.n_windows] == 0).all()
    n = w.n_hits
    np.testing.assert_array_equal(ext["ext_track"].cpu().numpy()[:n], ref["ext_track"].cpu().numpy()[:n])
    np.testing.assert_array_equal(ext["ext_hits"].cpu().numpy()[:n], ref["ext_hits"].cpu().numpy()[:n])
    f.close()
