"""The request loop (hough_server_*): each window's results are the same bits
whether its time slice runs alone or packed with others, admission and
back-pressure answer as documented, and every ticket is delivered once."""
import numpy as np
import pytest

from paper_2511_02742_gb300 import synth

pytestmark = pytest.mark.gpu


def _host_out(finder, n_windows, n_hits):
    return finder.alloc_outputs(n_windows, n_hits, device="cpu", pin=True)


def _reference(hough, finder, w):
    import torch
    hits = dict(vane=torch.from_numpy(w.vane).cuda(), strip=torch.from_numpy(w.strip).cuda())
    out = finder.find(hits, torch.from_numpy(w.offsets).cuda())
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


def _slices(w, sizes):
    """Contiguous window ranges of the given sizes, cycling over w."""
    out, a = [], 0
    for s in sizes:
        if a + s > w.n_windows:
            a = 0
        out.append((a, a + s))
        a += s
    return out


def _submit(srv, w, a, b, outs, arrival_ns=0):
    h0, h1 = int(w.offsets[a]), int(w.offsets[b])
    offs = (w.offsets[a:b + 1] - h0).astype(np.int64)
    o = {k: v for k, v in outs.items()}
    return srv.submit(w.vane[h0:h1], w.strip[h0:h1], offs, o, arrival_ns)


def _check(ref, w, a, b, out, max_peaks):
    h0, h1 = int(w.offsets[a]), int(w.offsets[b])
    got = {k: v.numpy() for k, v in out.items()}
    np.testing.assert_array_equal(got["n_peaks"], ref["n_peaks"][a:b])
    np.testing.assert_array_equal(got["n_found"], ref["n_found"][a:b])
    np.testing.assert_array_equal(got["window_status"], ref["window_status"][a:b])
    np.testing.assert_array_equal(got["hit_track"][:h1 - h0], ref["hit_track"][h0:h1])
    np.testing.assert_array_equal(got["track_hits"][:h1 - h0], ref["track_hits"][h0:h1])
    for j in range(b - a):
        n = int(ref["n_peaks"][a + j])
        np.testing.assert_array_equal(got["peaks"][j][:n], ref["peaks"][a + j][:n])


def test_results_same_alone_and_in_the_mix():
    from paper_2511_02742_gb300 import hough
    cfg = synth.WORKLOADS["serving"]
    w = synth.workload("serving", n_windows=600, seed=5)
    f = hough.Finder(cfg["n_theta"], cfg["n_rho"])
    ref = _reference(hough, f, w)
    srv = hough.Server(f, n_slots=2, slot_windows=256, slot_hits=1 << 17, max_queued=1024)
    try:
        # alone
        a, b = 100, 164
        out = _host_out(f, b - a, int(w.offsets[b] - w.offsets[a]))
        t = _submit(srv, w, a, b, out)
        r = srv.wait(t, 60000)
        assert r["status"] == 0 and r["batch_requests"] == 1
        _check(ref, w, a, b, out, f.max_peaks)
        # in the mix: 60 slices submitted back to back (the same slice among
        # them), so the queue builds up behind two slots and batches mix
        rng = np.random.default_rng(3)
        sizes = rng.integers(1, 40, size=60)
        sl = _slices(w, sizes)
        sl[30] = (a, b)
        outs = [_host_out(f, y - x, int(w.offsets[y] - w.offsets[x])) for (x, y) in sl]
        jobs = [(x, y, o, _submit(srv, w, x, y, o)) for (x, y), o in zip(sl, outs)]
        srv.drain(60000)
        results = {r["ticket"]: r for r in srv.poll(4096)}
        assert len(results) == len(jobs)
        assert max(r["batch_requests"] for r in results.values()) > 1
        for (x, y, o, t) in jobs:
            assert results[t]["status"] == 0
            _check(ref, w, x, y, o, f.max_peaks)
        st = srv.stats()
        assert st["completed"] == st["submitted"] == len(jobs) + 1
        assert st["queued"] == 0 and st["in_flight"] == 0
        assert st["windows"] == (b - a) + sum(y - x for (x, y, _, _) in jobs)
        assert st["batches"] < len(jobs) + 1
    finally:
        srv.close()
        f.close()


def test_encoded_hits_and_empty_windows():
    import torch
    from paper_2511_02742_gb300 import hough
    w = synth.workload("plain", n_windows=50, seed=2)
    # empty windows in the middle and at the end
    lens = np.diff(w.offsets)
    lens[[3, 4, 49]] = 0
    keep = np.concatenate([np.arange(w.offsets[k], w.offsets[k] + lens[k]) for k in range(50)])
    vane, strip = w.vane[keep], w.strip[keep]
    offs = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    f = hough.Finder(512, 512)
    phi = torch.empty(len(vane), dtype=torch.int32, device="cuda")
    z = torch.empty_like(phi)
    hough.hough_encode(f.ctx, torch.from_numpy(vane).cuda(), torch.from_numpy(strip).cuda(),
                       phi, z)
    ref = f.find(dict(phi_q=phi, z_q=z), torch.from_numpy(offs).cuda())
    torch.cuda.synchronize()
    ref = {k: v.cpu().numpy() for k, v in ref.items()}
    phi_h, z_h = phi.cpu().numpy(), z.cpu().numpy()
    srv = hough.Server(f, n_slots=1, slot_windows=64, slot_hits=1 << 16, raw_hits=False)
    try:
        out = _host_out(f, 50, len(vane))
        t = srv.submit(phi_h, z_h, offs, out)
        assert srv.wait(t, 60000)["status"] == 0
        got = {k: v.numpy() for k, v in out.items()}
        np.testing.assert_array_equal(got["n_peaks"], ref["n_peaks"])
        np.testing.assert_array_equal(got["hit_track"], ref["hit_track"])
        np.testing.assert_array_equal(got["track_hits"], ref["track_hits"])
        assert got["n_peaks"][3] == got["n_peaks"][4] == got["n_peaks"][49] == 0
        # a slice with no windows completes too
        t = srv.submit(phi_h[:0], z_h[:0], np.zeros(1, np.int64), _host_out(f, 0, 0))
        assert srv.wait(t, 60000)["status"] == 0
    finally:
        srv.close()
        f.close()


def test_admission_limits_and_errors():
    from paper_2511_02742_gb300 import hough
    w = synth.workload("batched", n_windows=6000, seed=4)
    f = hough.Finder(512, 512)
    srv = hough.Server(f, n_slots=1, slot_windows=2000, slot_hits=1 << 19, max_queued=1)
    try:
        out = _host_out(f, 2001, int(w.offsets[2001]))
        # more windows than a slot holds
        with pytest.raises(hough.HoughError) as e:
            _submit(srv, w, 0, 2001, out)
        assert e.value.code == hough.HOUGH_ERR_UNSUPPORTED_SHAPE
        # offsets not starting at 0 / decreasing
        bad = np.array([1, 5], np.int64)
        with pytest.raises(hough.HoughError) as e:
            srv.submit(w.vane, w.strip, bad, out)
        assert e.value.code == -1
        bad = np.array([0, 5, 4], np.int64)
        with pytest.raises(hough.HoughError):
            srv.submit(w.vane, w.strip, bad, out)
        # back-pressure: one slot busy with a 2000-window batch, one queued,
        # then BUSY
        busy, tickets = 0, []
        outs = [_host_out(f, 2000, int(w.offsets[(k + 1) * 2000] - w.offsets[k * 2000]))
                for k in range(3) for _ in range(4)]
        for k in range(3):
            for q in range(4):
                o = outs[4 * k + q]
                try:
                    tickets.append(_submit(srv, w, k * 2000, (k + 1) * 2000, o))
                except hough.HoughError as err:
                    assert err.code == hough.HOUGH_ERR_BUSY
                    busy += 1
        assert busy >= 1
        assert srv.stats()["rejected"] >= busy + 1
        for t in tickets:
            assert srv.wait(t, 60000)["status"] == 0
        # delivered once: a second wait on the same ticket is refused
        with pytest.raises(hough.HoughError):
            srv.wait(tickets[0], 0)
    finally:
        srv.close()
    # a context that exports accumulators cannot serve
    fe = hough.Finder(64, 64, export_acc=True)
    with pytest.raises(hough.HoughError):
        hough.Server(fe, n_slots=1, slot_windows=8, slot_hits=1024)
    fe.close()
    f.close()


def test_request_buffers_are_checked_before_submission():
    """The worker reads and writes a request through its pointers, so wrong
    types and short arrays are refused at submission."""
    from paper_2511_02742_gb300 import hough
    w = synth.workload("batched", n_windows=20, seed=5)
    f = hough.Finder(512, 512)
    srv = hough.Server(f, n_slots=1, slot_windows=64, slot_hits=1 << 16, max_queued=4)
    try:
        out = _host_out(f, 20, w.n_hits)
        with pytest.raises(TypeError):
            srv.submit(w.vane.astype(np.int64), w.strip, w.offsets, out)
        short = dict(out, hit_track=out["hit_track"][: w.n_hits - 1])
        with pytest.raises(ValueError):
            srv.submit(w.vane, w.strip, w.offsets, short)
        with pytest.raises(ValueError):
            srv.submit(w.vane[:-1], w.strip[:-1], w.offsets, out)
        t = srv.submit(w.vane, w.strip, w.offsets, out)
        assert srv.wait(t, 60000)["status"] == 0
    finally:
        srv.close()


def test_pageable_request_buffers():
    """Requests whose hits and result buffers are ordinary (pageable) host
    memory: the copies are staged by the driver, the results are the same."""
    from paper_2511_02742_gb300 import hough
    cfg = synth.WORKLOADS["serving"]
    w = synth.workload("serving", n_windows=120, seed=8)
    f = hough.Finder(cfg["n_theta"], cfg["n_rho"])
    ref = _reference(hough, f, w)
    srv = hough.Server(f, n_slots=2, slot_windows=256, slot_hits=1 << 18)
    vane, strip = w.vane.copy(), w.strip.copy()
    tickets = []
    for a, b in _slices(w, [40, 1, 79]):
        h0, h1 = int(w.offsets[a]), int(w.offsets[b])
        n = b - a
        out = {"peaks": np.zeros((n, f.max_peaks, 4), np.int32),
               "n_peaks": np.zeros(n, np.int32), "n_found": np.zeros(n, np.int32),
               "hit_track": np.zeros(max(h1 - h0, 1), np.int32),
               "track_hits": np.zeros(max(h1 - h0, 1), np.int32),
               "window_status": np.zeros(n, np.int32)}
        t = srv.submit(vane[h0:h1], strip[h0:h1], (w.offsets[a:b + 1] - h0).astype(np.int64), out)
        tickets.append((t, a, b, out))
    for t, a, b, out in tickets:
        assert srv.wait(t, 10000)["status"] == 0
        import torch
        _check(ref, w, a, b, {k: torch.from_numpy(v) for k, v in out.items()}, f.max_peaks)
    srv.close()
    f.close()


@pytest.mark.parametrize("tuned", [True, False])
def test_small_and_large_batches_under_the_default_shapes(tuned):
    """With the launch shape left open the server runs a batch of fewer than
    two windows per SM with one 1024-thread CTA per SM and a larger one with
    the context's shape (set, or left to the library, which picks it from the
    batch's hits per window); all give the bits hough_find gives, and the
    context's own shape is back after the server is closed."""
    import torch
    from paper_2511_02742_gb300 import hough
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    cfg = synth.WORKLOADS["serving"]
    w = synth.workload("serving", n_windows=4 * sms + 200, seed=12)
    f = hough.Finder(cfg["n_theta"], cfg["n_rho"])
    if tuned:
        hough.hough_set_launch(f.ctx, 512, 32, 1024, 2)
    before = hough.hough_get_launch(f.ctx)
    ref = _reference(hough, f, w)
    srv = hough.Server(f, n_slots=2, slot_windows=4 * sms + 200, slot_hits=1 << 21)
    try:
        jobs = []
        for a, b in [(0, 10), (10, 10 + 2 * sms + 50), (10 + 2 * sms + 50, 4 * sms + 200),
                     (5, 2 * sms + 4)]:
            out = _host_out(f, b - a, int(w.offsets[b] - w.offsets[a]))
            jobs.append((a, b, out, _submit(srv, w, a, b, out)))
            assert srv.wait(jobs[-1][3], 60000)["status"] == 0     # one request per batch
        for a, b, out, _ in jobs:
            _check(ref, w, a, b, out, f.max_peaks)
    finally:
        srv.close()
    assert hough.hough_get_launch(f.ctx) == before
    f.close()
