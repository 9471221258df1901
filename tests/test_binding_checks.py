"""The Python binding refuses buffers the kernels could misread: wrong dtype,
not contiguous, on the wrong side of the bus, or too small (no GPU needed:
the checks run before any call into the library)."""
import pytest
import torch

from paper_2511_02742_gb300 import hough


def test_buffer_checks():
    ok = torch.zeros(10, dtype=torch.int32)
    hough._check_buf(ok, torch.int32, 10, False, "x")
    with pytest.raises(TypeError):
        hough._check_buf(ok.numpy(), torch.int32, 1, False, "x")
    with pytest.raises(TypeError):
        hough._check_buf(ok.to(torch.int64), torch.int32, 1, False, "x")
    with pytest.raises(ValueError):
        hough._check_buf(torch.zeros((4, 4), dtype=torch.int32).t(), torch.int32, 1, False, "x")
    with pytest.raises(ValueError):
        hough._check_buf(ok, torch.int32, 11, False, "x")
    with pytest.raises(ValueError):
        hough._check_buf(ok, torch.int32, 1, True, "x")       # host tensor for a device call


def test_hits_and_outputs_checks():
    v = torch.zeros(5, dtype=torch.int32)
    assert hough._check_hits(dict(vane=v, strip=v), False) == 5
    with pytest.raises(ValueError):
        hough._check_hits(dict(vane=v, strip=torch.zeros(4, dtype=torch.int32)), False)
    i32 = torch.int32
    out = dict(peaks=torch.zeros((3, 8, 4), dtype=i32), n_peaks=torch.zeros(3, dtype=i32),
               n_found=None, window_status=torch.zeros(3, dtype=i32),
               hit_track=torch.zeros(5, dtype=i32), track_hits=torch.zeros(5, dtype=i32))
    hough._check_outputs(out, 3, 5, 8, None, False)
    with pytest.raises(ValueError):
        hough._check_outputs(out, 3, 5, 9, None, False)       # peaks too small for 9 per window
    with pytest.raises(ValueError):
        hough._check_outputs(out, 3, 6, 8, None, False)       # per-hit outputs too small
    with pytest.raises(TypeError):
        hough._check_outputs(out, 3, 5, 8, (4, 4), False)     # no accumulator given


def test_host_buffer_checks():
    import numpy as np
    hough._check_host(np.zeros(3, np.int32), np.int32, 3, "a")
    hough._check_host(torch.zeros(3, dtype=torch.int32), np.int32, 3, "b")
    for bad in (np.zeros(3, np.int64), torch.zeros(3, dtype=torch.int64), [1, 2, 3],
                np.zeros((3, 2), np.int32)[:, 0]):
        with pytest.raises(TypeError):
            hough._check_host(bad, np.int32, 1, "c")
    with pytest.raises(ValueError):
        hough._check_host(np.zeros(2, np.int32), np.int32, 3, "d")


def test_accumulate_checks_before_any_call():
    """Finder.accumulate refuses host hits and an accumulator too small for
    n_windows x n_theta x n_rho before it reaches the library."""
    import types
    stub = types.SimpleNamespace(n_theta=4, n_rho=8, ctx=None)
    v = torch.zeros(5, dtype=torch.int32)
    offs = torch.tensor([0, 2, 5], dtype=torch.int64)
    with pytest.raises(ValueError):
        hough.Finder.accumulate(stub, dict(vane=v, strip=v), offs)
    orig = hough._check_hits
    try:
        hough._check_hits = lambda hits, cuda: 5           # pretend the hits are on the GPU
        orig_buf = hough._check_buf
        seen = []

        def check_buf(x, dtype, n, cuda, name):
            seen.append((name, n))
            if name != "offsets":
                orig_buf(x, dtype, n, False, name)
        hough._check_buf = check_buf
        small = dict(acc=torch.zeros(2 * 4 * 8 - 1, dtype=torch.int32),
                     window_status=torch.zeros(2, dtype=torch.int32))
        with pytest.raises(ValueError):
            hough.Finder.accumulate(stub, dict(vane=v, strip=v), offs, out=small)
        assert ("acc", 2 * 4 * 8) in seen
    finally:
        hough._check_hits = orig
        hough._check_buf = orig_buf
