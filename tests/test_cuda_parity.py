"""Bit-exact parity of the CUDA path (through the C ABI) with the CPU oracle.

Everything here is integer, so the bar is exact equality of the accumulator
(export mode), the peak list, n_found, the window status, hit_track and
track_hits.
"""
import numpy as np
import pytest

import oracle
from paper_2511_02742_gb300 import synth
from parity_helpers import G, assert_batch_equal, assert_window_equal, gpu_run, oracle_run, to_numpy

pytestmark = pytest.mark.gpu


def _finder(hough, n_theta, n_rho, **kw):
    return hough.Finder(n_theta, n_rho, **kw)


@pytest.mark.parametrize("raw", [True, False])
def test_tiny_config_exact_with_accumulator(hough, raw):
    """10 single-track windows, 256 x 256, accumulator exported."""
    cfg = synth.WORKLOADS["tiny"]
    w = synth.workload("tiny")
    f = _finder(hough, cfg["n_theta"], cfg["n_rho"], export_acc=True)
    g = gpu_run(f, w, raw=raw)
    ref = oracle_run(w, cfg["n_theta"], cfg["n_rho"], export=True)
    assert_batch_equal(g, ref, w, check_acc=True)
    f.close()


def test_plain_config_exact(hough):
    """1000 windows x 5 tracks, 1% noise, 512 x 512: every window."""
    cfg = synth.WORKLOADS["plain"]
    w = synth.workload("plain")
    f = _finder(hough, cfg["n_theta"], cfg["n_rho"])
    g = gpu_run(f, w)
    ref = oracle_run(w, cfg["n_theta"], cfg["n_rho"])
    assert_batch_equal(g, ref, w)
    f.close()


def test_plain_config_accumulator_export(hough):
    cfg = synth.WORKLOADS["plain"]
    w = synth.workload("plain", n_windows=60, seed=1)
    f = _finder(hough, cfg["n_theta"], cfg["n_rho"], export_acc=True)
    g = gpu_run(f, w)
    ref = oracle_run(w, cfg["n_theta"], cfg["n_rho"], export=True)
    assert_batch_equal(g, ref, w, check_acc=True)
    f.close()


def test_high_pileup_sampled_windows(hough):
    """40 tracks/window, 5% noise, ~1e3 hits, 1024 x 1024: 300 windows on the
    GPU, 25 of them checked one by one against the oracle (accumulator too)."""
    cfg = synth.WORKLOADS["high_pileup"]
    w = synth.workload("high_pileup", n_windows=300)
    f = _finder(hough, cfg["n_theta"], cfg["n_rho"], export_acc=True)
    g = gpu_run(f, w)
    ids = np.random.default_rng(0).choice(w.n_windows, 25, replace=False)
    refs = oracle_run(w, cfg["n_theta"], cfg["n_rho"], export=True, ids=ids)
    for k, r in zip(ids, refs):
        assert_window_equal(g, int(k), r, w.window(int(k)), check_acc=True)
    f.close()


def test_uneven_batch_poisson(hough):
    """Poisson(10) tracks per window clipped to [1, 40], 2% noise, 512 x 512."""
    w = synth.generate(3000, ("poisson", 10, 1, 40), (100.0, 300.0), 0.02, seed=5)
    f = _finder(hough, 512, 512)
    g = gpu_run(f, w)
    ref = oracle_run(w, 512, 512)
    assert_batch_equal(g, ref, w)
    f.close()


@pytest.mark.parametrize("n_theta,n_rho", [(180, 1000), (97, 332), (33, 64), (1024, 256), (1, 4)])
def test_other_shapes(hough, n_theta, n_rho):
    """The paper's 180 x 1000 binning and ragged shapes (partial last tile)."""
    w = synth.generate(40, ("poisson", 8, 1, 40), (100.0, 300.0), 0.05, seed=n_theta)
    f = _finder(hough, n_theta, n_rho, export_acc=True)
    g = gpu_run(f, w)
    ref = oracle_run(w, n_theta, n_rho, export=True)
    assert_batch_equal(g, ref, w, check_acc=True)
    f.close()


def _windows_from_arrays(parts):
    """Windows from explicit (vane, strip) arrays."""
    vane = np.concatenate([np.asarray(p[0], np.int32) for p in parts]) if parts else np.zeros(0, np.int32)
    strip = np.concatenate([np.asarray(p[1], np.int32) for p in parts]) if parts else np.zeros(0, np.int32)
    off = np.zeros(len(parts) + 1, np.int64)
    off[1:] = np.cumsum([len(p[0]) for p in parts])
    n = len(vane)
    return synth.Windows(vane, strip, off, np.zeros(n, np.int32), np.zeros(n), np.zeros((0, 4)),
                         np.zeros(len(parts) + 1, np.int64))


def test_edge_cases(hough):
    """Empty windows, all hits at one point, hits on bin edges (phi = z = 0 sits
    on a rho edge in every row), out-of-range strip addresses, a window with
    fewer hits than T."""
    rng = np.random.default_rng(3)
    parts = [
        ([], []),
        ([5] * 40, [1000] * 40),                         # all hits at one (phi, z)
        ([0] * 12, [1024] * 12),                         # phi = 0, z at strip 1024 centre
        ([0, 1, 2], [7, 8, 9]),                          # < T hits
        ([40, 3, -1, 7, 7], [5, 2048, 0, -3, 100]),      # outside the detector box
        (rng.integers(0, 40, 300), rng.integers(0, 2048, 300)),
        ([], []),
    ]
    w = _windows_from_arrays(parts)
    for shape in [(256, 256), (180, 1000)]:
        f = _finder(hough, *shape, export_acc=True)
        g = gpu_run(f, w)
        ref = oracle_run(w, *shape, export=True)
        assert_batch_equal(g, ref, w, check_acc=True)
        f.close()


def test_encoded_hits_on_rho_edges(hough):
    """Encoded hits chosen so that many votes land exactly on a bin edge
    (floor of an exact integer quotient) and on the rho range ends."""
    phi = np.array([0, 0, 0, 36000, 71999, 1800, 0, 0], np.int32)
    z = np.array([0, 38912, -38912, 0, 0, 19, 1, -1], np.int32)
    import torch
    f = _finder(hough, 360, 1000, export_acc=True)
    hits = dict(phi_q=torch.from_numpy(phi).cuda(), z_q=torch.from_numpy(z).cuda())
    off = torch.tensor([0, len(phi)], dtype=torch.int64, device="cuda")
    out = f.find(hits, off)
    torch.cuda.synchronize()
    r = oracle.find_window(G, 360, 1000, phi, z)
    np.testing.assert_array_equal(out["acc"][0].cpu().numpy(), r["acc"])
    np.testing.assert_array_equal(out["hit_track"].cpu().numpy(), r["hit_track"])
    f.close()


def test_large_windows_multi_stage_and_wide_counters(hough):
    """A window larger than one shared-memory hit stage (16-bit counters, the
    hits streamed in stages) and one above 65535 hits (32-bit counters)."""
    rng = np.random.default_rng(7)
    parts = [(rng.integers(0, 40, 5000), rng.integers(0, 2048, 5000)),
             (rng.integers(0, 40, 70000), rng.integers(0, 2048, 70000)),
             (rng.integers(0, 40, 200), rng.integers(0, 2048, 200))]
    # make the big windows hold real peaks: add a few exact lines
    w = _windows_from_arrays(parts)
    f = _finder(hough, 128, 256, export_acc=True, vote_threshold=40, max_peaks=32)
    g = gpu_run(f, w)
    ref = oracle_run(w, 128, 256, export=True, vote_threshold=40, max_peaks=32)
    assert_batch_equal(g, ref, w, check_acc=True)
    f.close()


def test_peak_overflow_and_candidate_buffer_fallback(hough):
    """T = 1 on dense random windows: thousands of local maxima per tile
    overflow the candidate buffer and take the exact slice-by-slice path;
    the kept list must still be the exact top max_peaks."""
    rng = np.random.default_rng(11)
    parts = [(rng.integers(0, 40, 2000), rng.integers(0, 2048, 2000)) for _ in range(3)]
    w = _windows_from_arrays(parts)
    for mp in (256, 7, 0):
        ref = oracle_run(w, 256, 1024, vote_threshold=1, max_peaks=mp)
        assert ref["n_found"].min() > 3000
        f = _finder(hough, 256, 1024, vote_threshold=1, max_peaks=mp)
        ran = 0
        for lch in (None, (256, 32, 512, 3), (512, 32, 1024, 2), (1024, 32, 2048, 1),
                    (512, 32, 1024, 1), (256, 32, 256, 1)):
            if lch is not None:
                try:
                    hough.hough_set_launch(f.ctx, *lch)
                except hough.HoughError as e:
                    assert e.code == hough.HOUGH_ERR_UNSUPPORTED_SHAPE
                    continue
            assert_batch_equal(gpu_run(f, w), ref, w)
            ran += 1
        assert ran >= 3
        f.close()


def test_heavy_windows_in_small_ctas(hough):
    """Windows of 1 to 40 tracks (about 300 hits, half of them past the 8-bit
    limit) in three 256-thread CTAs per SM: the lists of some tiles overflow
    and those tiles take the direct test of every stored counter.  Equal to
    the oracle, in that shape and in larger ones."""
    cfg = synth.WORKLOADS["serving"]
    w = synth.workload("serving", n_windows=240, seed=4)
    ref = oracle_run(w, cfg["n_theta"], cfg["n_rho"])
    f = _finder(hough, cfg["n_theta"], cfg["n_rho"])
    for lch in (None, (256, 32, 512, 3), (256, 32, 1024, 3), (512, 32, 1024, 2),
                (1024, 32, 2048, 1)):
        if lch is not None:                     # None: the library's choice for heavy windows
            hough.hough_set_launch(f.ctx, *lch)
        assert_batch_equal(gpu_run(f, w), ref, w)
    f.close()


def test_bad_offsets_are_flagged_not_read(hough):
    import torch
    w = synth.generate(4, 3, (100.0, 300.0), 0.0, seed=1)
    f = _finder(hough, 64, 64)
    hits = dict(vane=torch.from_numpy(w.vane).cuda(), strip=torch.from_numpy(w.strip).cuda())
    off = w.offsets.copy()
    off[2] = off[1] - 1              # window 1 decreasing, window 2 starts before window 1 ends
    off_bad = np.concatenate([off, [w.n_hits + 10]])   # window 4 runs past n_hits
    offt = torch.from_numpy(off_bad).cuda()
    out = f.find(hits, offt)
    torch.cuda.synchronize()
    st = out["window_status"].cpu().numpy()
    assert st[1] & hough.HOUGH_WIN_BAD_OFFSETS
    assert st[4] & hough.HOUGH_WIN_BAD_OFFSETS
    assert not st[0] & hough.HOUGH_WIN_BAD_OFFSETS
    f.close()


def test_launch_shapes_identical(hough):
    """Every launch shape gives the same bits (deterministic integer path)."""
    w = synth.generate(300, ("poisson", 10, 1, 40), (100.0, 300.0), 0.02, seed=9)
    f = _finder(hough, 512, 512)
    base = gpu_run(f, w)
    shapes = [(t, wr, hs, 1) for t in (256, 512, 1024) for wr in (32, 64) for hs in (256, 2048)]
    shapes += [(256, 32, 1024, 3), (256, 32, 512, 3), (512, 32, 1024, 2), (256, 64, 512, 2)]
    for shape in shapes:
        hough.hough_set_launch(f.ctx, *shape)
        g = gpu_run(f, w)
        for k in ("n_peaks", "n_found", "status", "hit_track", "track_hits"):
            np.testing.assert_array_equal(g[k], base[k], err_msg=f"{k} {shape}")
        np.testing.assert_array_equal(g["peaks"], base["peaks"])
    f.close()


def test_narrowed_tiles_at_reach_edges(hough):
    """A tile stores only the bins that hits of the detector box can reach in
    its rows; the box's corners reach the extreme bins.  Stacks of hits at
    the four corners and hits along the box's edges (encoded, so the corners
    are exact), at several accumulator shapes and launch shapes (1 to 3 CTAs
    per SM, 32 to 128 word rows, a streamed stage): peaks, associations and the
    exported accumulator (zero outside the reachable bins) equal the
    oracle's."""
    import torch
    rng = np.random.default_rng(21)
    phi_hi = 360 * G["phi_u_per_deg"] - 1
    z_lo = G["z_min_u"]
    z_hi = G["z_min_u"] + G["n_z_strips"] * G["z_pitch_u"]
    corners = [(0, z_lo), (0, z_hi), (phi_hi, z_lo), (phi_hi, z_hi)]

    def stack(pts, n):
        return [p for p in pts for _ in range(n)]

    edge_phi = rng.integers(0, phi_hi + 1, 40)
    edge_z = rng.integers(z_lo, z_hi + 1, 40)
    wins = [
        stack(corners, 12),
        stack(corners[:1], 6) + stack(corners[3:], 9)
        + list(zip(rng.integers(0, phi_hi + 1, 50), rng.integers(z_lo, z_hi + 1, 50))),
        [(0, z) for z in edge_z] + [(p, z_hi) for p in edge_phi] + stack(corners[1:3], 7),
        stack(corners, 60) + [(p, z_lo) for p in edge_phi] + [(phi_hi, z) for z in edge_z],
        stack(corners, 5) + [(phi_hi + 1, 0), (0, z_hi + 1)],
    ]
    phi = np.array([p for wn in wins for p, _ in wn], np.int32)
    z = np.array([q for wn in wins for _, q in wn], np.int32)
    off = np.zeros(len(wins) + 1, np.int64)
    off[1:] = np.cumsum([len(wn) for wn in wins])
    assert off[4] - off[3] > 255                        # one window with 16-bit counters
    hits = dict(phi_q=torch.from_numpy(phi).cuda(), z_q=torch.from_numpy(z).cuda())
    offs = torch.from_numpy(off).cuda()
    launches = [None, (256, 32, 1024, 3), (512, 32, 1024, 2), (1024, 32, 2048, 1),
                (512, 64, 1024, 1), (512, 128, 1024, 1), (256, 32, 256, 1)]
    for n_theta, n_rho in [(512, 512), (1024, 1024), (180, 1000), (97, 332), (128, 512), (33, 64)]:
        ref = oracle.find_batch(G, n_theta, n_rho, phi, z, off, export_acc=True)
        assert ref["status"][4] & hough.HOUGH_WIN_HIT_OUT_OF_RANGE
        f = _finder(hough, n_theta, n_rho, export_acc=True)
        ran = 0
        for lch in launches:
            if lch is not None:
                try:
                    hough.hough_set_launch(f.ctx, *lch)
                except hough.HoughError as e:
                    assert e.code == hough.HOUGH_ERR_UNSUPPORTED_SHAPE
                    continue
            out = f.find(hits, offs)
            torch.cuda.synchronize()
            g = to_numpy(out, len(phi))
            wn = synth.Windows(phi, z, off, np.zeros(len(phi), np.int32), np.zeros(len(phi)),
                               np.zeros((0, 4)), np.zeros(len(wins) + 1, np.int64))
            assert_batch_equal(g, ref, wn, check_acc=True)
            ran += 1
        assert ran >= 3, (n_theta, n_rho, ran)
        f.close()


def test_alone_vs_batch_and_repeat(hough):
    """A window gives the same result alone (one window per call) and inside a
    batch, and a repeated run gives the same bits."""
    import torch
    w = synth.generate(50, ("poisson", 10, 1, 40), (100.0, 300.0), 0.02, seed=12)
    f = _finder(hough, 512, 512)
    a = gpu_run(f, w)
    b = gpu_run(f, w)
    for k in a:
        np.testing.assert_array_equal(a[k], b[k])
    hits = dict(vane=torch.from_numpy(w.vane).cuda(), strip=torch.from_numpy(w.strip).cuda())
    offs = torch.from_numpy(w.offsets).cuda()
    out = f.alloc_outputs(w.n_windows, w.n_hits)
    for k in range(w.n_windows):
        sub = {key: (v[k:k + 1] if key in ("peaks", "n_peaks", "n_found", "window_status") else v)
               for key, v in out.items()}
        hough.hough_find(f.ctx, f.hits_struct(hits), offs[k:k + 2], 1, hough.make_tracks(sub))
    torch.cuda.synchronize()
    from parity_helpers import to_numpy
    c = to_numpy(out, w.n_hits)
    for k in a:
        np.testing.assert_array_equal(a[k], c[k], err_msg=k)
    f.close()


def test_plan_graph_and_host_entry_point(hough):
    """The CUDA-graph plan and the host-buffer entry point give the same bits."""
    import torch
    w = synth.generate(500, ("poisson", 10, 1, 40), (100.0, 300.0), 0.02, seed=13)
    f = _finder(hough, 512, 512)
    a = gpu_run(f, w)
    hits = dict(vane=torch.from_numpy(w.vane).cuda(), strip=torch.from_numpy(w.strip).cuda())
    offs = torch.from_numpy(w.offsets).cuda()
    out = f.alloc_outputs(w.n_windows, w.n_hits)
    plan = f.plan(hits, offs, out)
    for _ in range(3):
        hough.hough_plan_launch(plan)
    torch.cuda.synchronize()
    from parity_helpers import to_numpy
    b = to_numpy(out, w.n_hits)
    for k in a:
        np.testing.assert_array_equal(a[k], b[k], err_msg=k)
    hough.hough_plan_destroy(plan)
    hh = dict(vane=torch.from_numpy(w.vane).pin_memory(), strip=torch.from_numpy(w.strip).pin_memory())
    oh = f.alloc_outputs(w.n_windows, w.n_hits, device="cpu", pin=True)
    f.find_host(hh, torch.from_numpy(w.offsets), out=oh)
    c = to_numpy(oh, w.n_hits)
    for k in a:
        np.testing.assert_array_equal(a[k], c[k], err_msg=k)
    f.close()


def test_host_entry_point_in_chunks_with_export(hough):
    """hough_find_host over 9000 windows (copies and kernels pipelined in
    chunks over two streams), empty windows included, accumulators exported:
    the same bits as the device entry point."""
    import torch
    w = synth.generate(9000, ("poisson", 4, 0, 12), (100.0, 300.0), 0.02, seed=21)
    f = _finder(hough, 64, 128, export_acc=True)
    a = gpu_run(f, w)
    hh = dict(vane=torch.from_numpy(w.vane).pin_memory(), strip=torch.from_numpy(w.strip).pin_memory())
    oh = f.alloc_outputs(w.n_windows, w.n_hits, device="cpu", pin=True)
    for v in oh.values():
        v.fill_(-3)
    f.find_host(hh, torch.from_numpy(w.offsets), out=oh)
    c = to_numpy(oh, w.n_hits)
    assert (np.diff(w.offsets) == 0).any()
    for k in ("n_peaks", "n_found", "hit_track", "track_hits", "status", "acc"):
        np.testing.assert_array_equal(a[k], c[k], err_msg=k)
    for k in range(w.n_windows):
        n = int(a["n_peaks"][k])
        np.testing.assert_array_equal(a["peaks"][k][:n], c["peaks"][k][:n])
    f.close()


def test_autotune_keeps_results(hough):
    import torch
    w = synth.generate(400, ("poisson", 10, 1, 40), (100.0, 300.0), 0.02, seed=14)
    f = _finder(hough, 512, 512)
    a = gpu_run(f, w)
    hits = dict(vane=torch.from_numpy(w.vane).cuda(), strip=torch.from_numpy(w.strip).cuda())
    offs = torch.from_numpy(w.offsets).cuda()
    out = f.alloc_outputs(w.n_windows, w.n_hits)
    best = f.autotune(hits, offs, out, iters=1)
    torch.cuda.synchronize()
    assert best["threads"] in (256, 512, 1024)
    from parity_helpers import to_numpy
    b = to_numpy(out, w.n_hits)
    for k in a:
        np.testing.assert_array_equal(a[k], b[k], err_msg=k)
    f.close()


def test_encode_entry_point(hough):
    import torch
    w = synth.generate(20, 5, (100.0, 300.0), 0.05, seed=2)
    f = _finder(hough, 64, 64)
    vane = torch.from_numpy(np.concatenate([w.vane, [40, -1]]).astype(np.int32)).cuda()
    strip = torch.from_numpy(np.concatenate([w.strip, [2048, -5]]).astype(np.int32)).cuda()
    phi = torch.empty_like(vane)
    z = torch.empty_like(vane)
    hough.hough_encode(f.ctx, vane, strip, phi, z)
    torch.cuda.synchronize()
    rp, rz = oracle.encode(G, vane.cpu().numpy(), strip.cpu().numpy())
    np.testing.assert_array_equal(phi.cpu().numpy(), rp)
    np.testing.assert_array_equal(z.cpu().numpy(), rz)
    f.close()


def test_export_to_an_unaligned_accumulator(hough):
    """An accumulator pointer that is not 16-byte aligned gets the same values
    (the kernel then writes 4-byte words instead of 16-byte vectors)."""
    import torch
    w = synth.generate(30, ("poisson", 10, 1, 40), (100.0, 300.0), 0.02, seed=41)
    f = _finder(hough, 96, 332, export_acc=True)
    hits = dict(vane=torch.from_numpy(w.vane).cuda(), strip=torch.from_numpy(w.strip).cuda())
    offs = torch.from_numpy(w.offsets).cuda()
    a = f.find(hits, offs)
    out = f.alloc_outputs(w.n_windows, w.n_hits)
    buf = torch.full((w.n_windows * 96 * 332 + 1,), -5, dtype=torch.int32, device="cuda")
    out["acc"] = buf[1:].view(w.n_windows, 96, 332)
    assert out["acc"].data_ptr() % 16 == 4
    f.find(hits, offs, out=out)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(out["acc"].cpu().numpy(), a["acc"].cpu().numpy())
    assert int(buf[0].item()) == -5
    f.close()


@pytest.mark.parametrize("shift_a,shift_b", [(0, 0), (1, 1), (2, 3), (0, 1)])
def test_hit_arrays_at_any_alignment(hough, shift_a, shift_b):
    """Windows of 0 to about 80 hits starting at every residue mod 4, with the
    hit arrays 16-byte aligned or shifted by 4 to 12 bytes (each array on its
    own): every window equals the oracle's, for encoded hits and raw ones."""
    import torch
    rng = np.random.default_rng(77)
    parts = [synth.generate(1, int(rng.integers(0, 4)), (100.0, 300.0), float(rng.uniform(0, 0.05)),
                            seed=700 + k) for k in range(160)]
    w = synth.concat(parts)
    n = np.diff(w.offsets)
    assert set(w.offsets[:-1][n >= 8] % 4) == {0, 1, 2, 3} and (n == 0).any() and (n < 4).any()
    f = _finder(hough, 256, 256)
    phi, z = oracle.encode(f.geometry, w.vane, w.strip)
    ref = oracle_run(w, 256, 256)
    for raw in (True, False):
        a, b = (w.vane, w.strip) if raw else (phi, z)
        ta = torch.zeros(len(a) + 4, dtype=torch.int32, device="cuda")
        tb = torch.zeros(len(b) + 4, dtype=torch.int32, device="cuda")
        va, vb = ta[shift_a:shift_a + len(a)], tb[shift_b:shift_b + len(b)]
        va.copy_(torch.from_numpy(a))
        vb.copy_(torch.from_numpy(b))
        assert va.data_ptr() % 16 == 4 * shift_a and vb.data_ptr() % 16 == 4 * shift_b
        hits = dict(vane=va, strip=vb) if raw else dict(phi_q=va, z_q=vb)
        out = f.find(hits, torch.from_numpy(w.offsets).cuda())
        torch.cuda.synchronize()
        assert_batch_equal(to_numpy(out, w.n_hits), ref, w)
    f.close()


def test_windows_around_the_8bit_counter_limit(hough):
    """Windows on both sides of the 255-hit limit of 8-bit counters: 255
    stacked hits (8-bit, a bin of 255), 300 and 256+100 hits (16-bit, bins
    of 300 and 256), 400 random hits.  Equal to the oracle, accumulators
    included."""
    rng = np.random.default_rng(9)
    parts = [([7] * 300, [1500] * 300),
             (rng.integers(0, 40, 400), rng.integers(0, 2048, 400)),
             ([3] * 255, [100] * 255),
             (np.r_[[9] * 255, rng.integers(0, 40, 100)], np.r_[[700] * 255, rng.integers(0, 2048, 100)]),
             (np.r_[[9] * 256, rng.integers(0, 40, 100)], np.r_[[700] * 256, rng.integers(0, 2048, 100)])]
    w = _windows_from_arrays(parts)
    for export in (False, True):
        ref = oracle_run(w, 128, 512, export=export)
        assert ref["peaks"][0][0]["votes"] == 300
        f = _finder(hough, 128, 512, export_acc=export)
        assert_batch_equal(gpu_run(f, w), ref, w, check_acc=export)
        f.close()
