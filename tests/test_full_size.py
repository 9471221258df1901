"""Parity at the full benchmark sizes, in the launch configuration the bench
times (autotuned shape, CUDA-graph plan): the batched workload (1e5 windows,
512 x 512) and the high-pileup workload (1e4 windows, 1024 x 1024, exported
accumulators), each checked against the oracle window by window on a
seeded sample."""
import numpy as np
import pytest

import oracle
from paper_2511_02742_gb300 import synth
from parity_helpers import G, assert_window_equal, to_numpy

pytestmark = pytest.mark.gpu


TOL_Z = 16 * 38


def _run_planned(hough, w, n_theta, n_rho, export=False, tune_windows=20000, extend=False):
    import torch
    f = hough.Finder(n_theta, n_rho, export_acc=export)
    hits = dict(vane=torch.from_numpy(w.vane).cuda(), strip=torch.from_numpy(w.strip).cuda())
    offs = torch.from_numpy(w.offsets).cuda()
    sub = w.subset(np.arange(min(w.n_windows, tune_windows)))
    sh = dict(vane=torch.from_numpy(sub.vane).cuda(), strip=torch.from_numpy(sub.strip).cuda())
    f.autotune(sh, torch.from_numpy(sub.offsets).cuda(),
               f.alloc_outputs(sub.n_windows, sub.n_hits), iters=1)
    out = f.alloc_outputs(w.n_windows, w.n_hits)
    plan = f.plan(hits, offs, out)
    for _ in range(2):
        hough.hough_plan_launch(plan)
    torch.cuda.synchronize()
    hough.hough_plan_destroy(plan)
    launch = hough.hough_get_launch(f.ctx)
    if extend:
        out["ext"] = f.extend(hits, offs, out, TOL_Z)
        torch.cuda.synchronize()
    f.close()
    return out, launch


def test_batched_full_size_sampled(hough):
    cfg = synth.WORKLOADS["batched"]
    w = synth.workload("batched")
    assert w.n_windows == 100000
    out, launch = _run_planned(hough, w, cfg["n_theta"], cfg["n_rho"], extend=True)
    ext = out.pop("ext")
    g = to_numpy(out, w.n_hits)
    ids = np.random.default_rng(2).choice(w.n_windows, 60, replace=False)
    refs = oracle_windows(w, ids, cfg["n_theta"], cfg["n_rho"])
    from paper_2511_02742_gb300 import hough as hb
    et = ext["tracks"].cpu().numpy().view(hb.EXT_DTYPE).reshape(w.n_windows, -1)
    ex_track = ext["ext_track"].cpu().numpy()
    ex_hits = ext["ext_hits"].cpu().numpy()
    assert (ext["window_status"].cpu().numpy()[:w.n_windows] == 0).all()
    for k, r in zip(ids, refs):
        sl = w.window(int(k))
        assert_window_equal(g, int(k), r, sl, check_acc=False)
        re, rt, rh = oracle_extend_window(w, int(k), r)
        np.testing.assert_array_equal(et[int(k)][:r["n_peaks"]], re[0][:r["n_peaks"]])
        np.testing.assert_array_equal(ex_track[sl], rt)
        np.testing.assert_array_equal(ex_hits[sl], rh)


def test_high_pileup_full_size_sampled_with_accumulators(hough):
    import torch
    cfg = synth.WORKLOADS["high_pileup"]
    w = synth.workload("high_pileup")
    assert w.n_windows == 10000
    out, launch = _run_planned(hough, w, cfg["n_theta"], cfg["n_rho"], export=True,
                               tune_windows=500)
    g = to_numpy({k: v for k, v in out.items() if k != "acc"}, w.n_hits)
    ids = np.random.default_rng(3).choice(w.n_windows, 12, replace=False)
    refs = oracle_windows(w, ids, cfg["n_theta"], cfg["n_rho"], export=True)
    for k, r in zip(ids, refs):
        assert_window_equal(g, int(k), r, w.window(int(k)), check_acc=False)
        np.testing.assert_array_equal(out["acc"][int(k)].cpu().numpy(), r["acc"])


def oracle_windows(w, ids, n_theta, n_rho, export=False):
    phi, z = oracle.encode(G, w.vane, w.strip)
    res = []
    for k in ids:
        sl = w.window(int(k))
        res.append(oracle.find_window(G, n_theta, n_rho, phi[sl], z[sl]))
    return res


def oracle_extend_window(w, k, r, max_peaks=64):
    """The oracle's track extension of window k from its own step A-D result r."""
    sl = w.window(k)
    phi, z = oracle.encode(G, w.vane[sl], w.strip[sl])
    pk = np.zeros((1, max_peaks), oracle.PEAK_DTYPE)
    pk[0, :r["n_peaks"]] = r["peaks"]
    found = dict(peaks=pk, n_peaks=np.array([r["n_peaks"]], np.int32), hit_track=r["hit_track"],
                 track_hits=r["track_hits"])
    return oracle.extend(G, phi, z, np.array([0, sl.stop - sl.start], np.int64), found, TOL_Z)
