"""hough_accumulate (steps A-B, every window's accumulator written out)
against the oracle's accumulator, bit-exact, and against the accumulator the
find step exports: the per-window histograms of Eq. (1) with the Section 5
binning, and the per-window status bits for rejected hits, votes outside the
rho range and bad offsets."""
import numpy as np
import pytest

import oracle
from paper_2511_02742_gb300 import synth
from parity_helpers import G

pytestmark = pytest.mark.gpu
FLAGS = 2 | 4 | 8       # HIT_OUT_OF_RANGE, VOTE_OUT_OF_RANGE, BAD_OFFSETS


def _hits(w, raw, phi=None, z=None):
    import torch
    if raw:
        return dict(vane=torch.from_numpy(w.vane).cuda(), strip=torch.from_numpy(w.strip).cuda())
    return dict(phi_q=torch.from_numpy(phi).cuda(), z_q=torch.from_numpy(z).cuda())


def _run(hough, w, n_theta, n_rho, raw=True, phi=None, z=None, geom=G):
    import torch
    f = hough.Finder(n_theta, n_rho, geometry=geom)
    out = f.accumulate(_hits(w, raw, phi, z), torch.from_numpy(w.offsets).cuda())
    torch.cuda.synchronize()
    r = out["acc"].cpu().numpy(), out["window_status"].cpu().numpy()[:w.n_windows].astype(np.uint32)
    f.close()
    return r


def _oracle(w, n_theta, n_rho, phi=None, z=None, geom=G):
    if phi is None:
        phi, z = oracle.encode(geom, w.vane, w.strip)
    r = oracle.find_batch(geom, n_theta, n_rho, phi, z, w.offsets, export_acc=True, max_peaks=1)
    return r["acc"], r["status"] & FLAGS


def _check(hough, w, n_theta, n_rho, raw=True, phi=None, z=None, geom=G):
    ga, gs = _run(hough, w, n_theta, n_rho, raw, phi, z, geom)
    ra, rs = _oracle(w, n_theta, n_rho, phi, z, geom)
    np.testing.assert_array_equal(gs, rs)
    for k in range(w.n_windows):
        np.testing.assert_array_equal(ga[k], ra[k], err_msg=f"window {k}")
    return ga, gs


@pytest.mark.parametrize("raw", [True, False])
def test_tiny_and_plain(hough, raw):
    for name, n in (("tiny", None), ("plain", 120)):
        w = synth.workload(name, n_windows=n, seed=81)
        cfg = synth.WORKLOADS[name]
        phi, z = oracle.encode(G, w.vane, w.strip)
        ga, _ = _check(hough, w, cfg["n_theta"], cfg["n_rho"], raw, phi, z)
        assert ga.sum() > 0


def test_high_pileup_windows(hough):
    """About 10^3 hits per window at 1024 x 1024 (16-bit counters, one CTA of
    1024 threads per SM)."""
    w = synth.workload("high_pileup", n_windows=12, seed=82)
    assert np.diff(w.offsets).min() > 255
    _check(hough, w, 1024, 1024)


def test_uneven_windows_every_counter_width(hough):
    """Empty windows, windows under and over 255 hits, one over the 2048-hit
    stage (streamed in parts) and one over 65535 hits (32-bit counters),
    interleaved."""
    rng = np.random.default_rng(83)
    base = synth.concat([synth.generate(40, ("poisson", 10, 0, 40), (100.0, 300.0), 0.02, seed=84),
                         synth.generate(4, 0, (100.0, 300.0), 0.0, seed=85)])
    parts = [(base.vane[base.window(k)], base.strip[base.window(k)]) for k in range(base.n_windows)]
    parts.insert(7, (rng.integers(0, 40, 5000), rng.integers(0, 2048, 5000)))
    parts.insert(20, (rng.integers(0, 40, 70000), rng.integers(0, 2048, 70000)))
    parts.insert(30, (rng.integers(0, 40, 1000), rng.integers(0, 2048, 1000)))
    vane = np.concatenate([np.asarray(p[0], np.int32) for p in parts])
    strip = np.concatenate([np.asarray(p[1], np.int32) for p in parts])
    off = np.zeros(len(parts) + 1, np.int64)
    off[1:] = np.cumsum([len(p[0]) for p in parts])
    n = len(vane)
    w = synth.Windows(vane, strip, off, np.zeros(n, np.int32), np.zeros(n), np.zeros((0, 4)),
                      np.zeros(len(parts) + 1, np.int64))
    sizes = np.diff(off)
    assert (sizes == 0).any() and (sizes <= 255).any() and ((sizes > 255) & (sizes <= 2048)).any()
    assert (sizes > 2048).any() and (sizes > 65535).any()
    _check(hough, w, 128, 256)


@pytest.mark.parametrize("n_theta,n_rho", [(97, 332), (33, 64), (1, 4), (1024, 256), (180, 1000)])
def test_other_shapes(hough, n_theta, n_rho):
    w = synth.generate(30, ("poisson", 6, 1, 30), (100.0, 300.0), 0.02, seed=86)
    _check(hough, w, n_theta, n_rho)


def test_rejected_hits_and_votes_out_of_range(hough):
    """Encoded hits off the detector box are rejected (HIT_OUT_OF_RANGE);
    with a narrow rho range, votes fall outside it (VOTE_OUT_OF_RANGE)."""
    w = synth.generate(40, ("poisson", 8, 1, 30), (100.0, 300.0), 0.02, seed=87)
    phi, z = oracle.encode(G, w.vane, w.strip)
    rng = np.random.default_rng(87)
    k = rng.choice(w.n_hits, w.n_hits // 30, replace=False)
    z[k] = 10 ** 6
    _, gs = _check(hough, w, 256, 256, raw=False, phi=phi, z=z)
    assert (gs & 2).any()
    narrow = dict(G, rho_min=-100.0, rho_max=100.0)
    _, gs = _check(hough, w, 256, 256, raw=False, phi=phi, z=z, geom=narrow)
    assert (gs & 4).any()


def test_equals_the_find_export(hough):
    """The same accumulators as hough_find with HOUGH_FLAG_EXPORT_ACC."""
    import torch
    w = synth.workload("batched", n_windows=300, seed=88)
    f = hough.Finder(512, 512, export_acc=True)
    hits = _hits(w, True)
    offs = torch.from_numpy(w.offsets).cuda()
    a = f.find(hits, offs)
    b = f.accumulate(hits, offs)
    torch.cuda.synchronize()
    assert torch.equal(a["acc"], b["acc"])
    assert torch.equal(a["window_status"] & FLAGS, b["window_status"][:w.n_windows])
    f.close()


def test_unaligned_accumulator_and_bad_offsets(hough):
    """An accumulator that is not 16-byte aligned gets the same values; a
    window whose offsets run backwards or past the hits is flagged and its
    accumulator is left as it was."""
    import torch
    w = synth.generate(20, ("poisson", 8, 1, 30), (100.0, 300.0), 0.02, seed=89)
    f = hough.Finder(96, 332)
    hits = _hits(w, True)
    ref = f.accumulate(hits, torch.from_numpy(w.offsets).cuda())
    bad = np.concatenate([w.offsets, [w.offsets[-1] + 1000, w.offsets[2]]])
    nw = len(bad) - 1
    buf = torch.full((nw * 96 * 332 + 1,), -5, dtype=torch.int32, device="cuda")
    out = dict(acc=buf[1:].view(nw, 96, 332),
               window_status=torch.full((nw,), -7, dtype=torch.int32, device="cuda"))
    assert out["acc"].data_ptr() % 16 == 4
    f.accumulate(hits, torch.from_numpy(bad).cuda(), out=out)
    torch.cuda.synchronize()
    assert torch.equal(out["acc"][:w.n_windows], ref["acc"])
    assert (out["acc"][w.n_windows:] == -5).all() and int(buf[0].item()) == -5
    st = out["window_status"].cpu().numpy()
    assert list(st[w.n_windows:]) == [8, 8]
    assert torch.equal(out["window_status"][:w.n_windows], ref["window_status"][:w.n_windows])
    f.close()


def test_fp64_context_is_rejected(hough):
    import torch
    f = hough.Finder(64, 64, fp64=True)
    w = synth.workload("tiny")
    with pytest.raises(hough.HoughError) as e:
        f.accumulate(_hits(w, True), torch.from_numpy(w.offsets).cuda())
    assert e.value.code == -1
    f.close()
