"""The FP64 variant of the find kernel (HOUGH_FLAG_FP64) against the
oracle's FP64 variant, bit-exact: both evaluate Eq. (1) in double precision
with the same correctly rounded operations in the same order, so the
accumulator, the peaks and the association are identical.  And the
within-one-bin agreement of the FP64 and fixed-point finds on the GPU."""
import numpy as np
import pytest

import oracle
from paper_2511_02742_gb300 import synth
from parity_helpers import G, assert_batch_equal, gpu_run, oracle_run

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("raw", [True, False])
def test_tiny_with_accumulator(hough, raw):
    w = synth.workload("tiny")
    f = hough.Finder(256, 256, export_acc=True, fp64=True)
    g = gpu_run(f, w, raw=raw)
    ref = oracle_run(w, 256, 256, export=True, fp64=True)
    assert_batch_equal(g, ref, w, check_acc=True)
    f.close()


@pytest.mark.parametrize("shape", [(512, 512), (180, 1000), (97, 332)])
def test_pileup_windows(hough, shape):
    w = synth.generate(150, ("poisson", 10, 0, 40), (100.0, 300.0), 0.02, seed=31)
    f = hough.Finder(*shape, export_acc=True, fp64=True)
    g = gpu_run(f, w)
    ref = oracle_run(w, *shape, export=True, fp64=True)
    assert_batch_equal(g, ref, w, check_acc=True)
    f.close()


def test_high_pileup_and_large_windows(hough):
    """16-bit counters (high pileup at 1024 x 1024) and 32-bit counters (a
    window above 65535 hits), both through the FP64 bins."""
    w = synth.workload("high_pileup", n_windows=3, seed=32)
    f = hough.Finder(1024, 1024, fp64=True)
    assert_batch_equal(gpu_run(f, w), oracle_run(w, 1024, 1024, fp64=True), w)
    f.close()
    big = synth.generate(1, 2500, (100.0, 300.0), 1.0, seed=33)
    assert big.n_hits > 65535
    f = hough.Finder(48, 128, fp64=True)
    assert_batch_equal(gpu_run(f, big), oracle_run(big, 48, 128, fp64=True), big)
    f.close()


def test_arbitrary_encoded_hits(hough):
    """Encoded hits anywhere in the box (phi off the vane angles), some outside."""
    import torch
    rng = np.random.default_rng(34)
    n = 4000
    phi = rng.integers(-500, 360 * 200 + 500, n).astype(np.int32)
    z = rng.integers(-39500, 39500, n).astype(np.int32)
    offsets = np.array([0, 700, 700, 2500, 4000], np.int64)
    f = hough.Finder(256, 512, fp64=True)
    out = f.find(dict(phi_q=torch.from_numpy(phi).cuda(), z_q=torch.from_numpy(z).cuda()),
                 torch.from_numpy(offsets).cuda())
    torch.cuda.synchronize()
    ref = oracle.find_batch(G, 256, 512, phi, z, offsets, fp64=True)
    from parity_helpers import to_numpy

    class W:
        n_windows = len(offsets) - 1
    assert_batch_equal(to_numpy(out, n), ref, W)
    f.close()


def test_fp64_and_fixed_agree_within_one_bin(hough):
    """On the GPU: the FP64 top peak lies within one bin of a fixed-point peak
    holding at least the fixed-point top count minus one."""
    w = synth.generate(300, ("poisson", 10, 1, 40), (100.0, 300.0), 0.02, seed=35)
    a = gpu_run(hough.Finder(512, 512), w)
    b = gpu_run(hough.Finder(512, 512, fp64=True), w)
    n = 0
    for k in range(w.n_windows):
        if a["n_peaks"][k] == 0 or a["peaks"][k][0]["votes"] < 10:
            continue
        n += 1
        pa = a["peaks"][k][:a["n_peaks"][k]]
        pb = b["peaks"][k][0]
        near = pa[pa["votes"] >= int(pa[0]["votes"]) - 1]
        assert ((np.abs(near["theta"].astype(int) - int(pb["theta"])) <= 1) &
                (np.abs(near["rho"].astype(int) - int(pb["rho"])) <= 1)).any(), k
    assert n > 200


def test_no_alloc_entry_refuses_the_flag(hough):
    import torch
    w = synth.workload("tiny")
    f = hough.Finder(64, 64)
    out = f.alloc_outputs(w.n_windows, w.n_hits)
    hits = f.hits_struct(dict(vane=torch.from_numpy(w.vane).cuda(),
                              strip=torch.from_numpy(w.strip).cuda()))
    with pytest.raises(hough.HoughError) as e:
        hough.hough_find_noalloc(G, 64, 64, hits, torch.from_numpy(w.offsets).cuda(),
                                 w.n_windows, hough.make_tracks(out), flags=hough.HOUGH_FLAG_FP64)
    assert e.value.code == -1
    f.close()
