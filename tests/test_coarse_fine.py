"""The coarse-to-fine kernel (the paper's two-stage GPU search) against the
oracle, bit-exact: per-window coarse and fine maxima, seeds and hit_track."""
import numpy as np
import pytest

import oracle
from paper_2511_02742_gb300 import synth

pytestmark = pytest.mark.gpu
G = synth.GEOMETRY


def _gpu(hough, w, raw=True, f=None):
    import torch
    own = f is None
    f = f or hough.Finder(512, 512)
    if raw:
        hits = dict(vane=torch.from_numpy(w.vane).cuda(), strip=torch.from_numpy(w.strip).cuda())
    else:
        phi, z = oracle.encode(G, w.vane, w.strip)
        hits = dict(phi_q=torch.from_numpy(phi).cuda(), z_q=torch.from_numpy(z).cuda())
    lines = torch.full((w.n_windows, 8), -7, dtype=torch.int32, device="cuda")
    ht = torch.full((max(w.n_hits, 1),), -7, dtype=torch.int32, device="cuda")
    hough.hough_find_coarse_fine(f.ctx, f.hits_struct(hits), torch.from_numpy(w.offsets).cuda(),
                                 w.n_windows, lines, ht)
    torch.cuda.synchronize()
    if own:
        f.close()
    return lines.cpu().numpy().view(hough.LINE_DTYPE).reshape(-1), ht.cpu().numpy()[:w.n_hits]


def _check(hough, w, raw=True):
    g, ght = _gpu(hough, w, raw)
    phi, z = oracle.encode(G, w.vane, w.strip)
    r, rht = oracle.coarse_fine(G, phi, z, w.offsets)
    for name in oracle.CF_DTYPE.names:
        np.testing.assert_array_equal(g[name], r[name], err_msg=name)
    np.testing.assert_array_equal(ght, rht)


@pytest.mark.parametrize("raw", [True, False])
def test_plain_workload(hough, raw):
    _check(hough, synth.workload("plain", n_windows=400, seed=3), raw)


def test_uneven_windows_and_high_pileup(hough):
    _check(hough, synth.generate(2000, ("poisson", 10, 0, 40), (100.0, 300.0), 0.02, seed=4))
    _check(hough, synth.workload("high_pileup", n_windows=60, seed=5))


def test_lines_and_edge_windows(hough):
    parts = [synth.line_window(84.5, 5.5), synth.line_window(104.5, 3.5),
             synth.generate(3, 0, (100.0, 300.0), 0.0, seed=1)]
    w = synth.concat(parts)
    g, ght = _gpu(hough, w)
    assert (g["fine_theta"][0], g["fine_rho"][0]) == (84, 505)
    assert (g["fine_theta"][1], g["fine_rho"][1]) == (104, 503)
    assert (g["found"][2:] == 0).all()
    _check(hough, w)


def test_tables_survive_host_entry_point_staging(hough):
    """The two-stage search keeps its tables in the context; the host-buffer
    find growing its device staging afterwards must leave them in place: the
    same context gives the same lines before and after."""
    import torch
    w = synth.workload("plain", n_windows=200, seed=8)
    f = hough.Finder(512, 512)
    a, aht = _gpu(hough, w, f=f)
    big = synth.generate(3000, ("poisson", 10, 1, 40), (100.0, 300.0), 0.02, seed=9)
    hh = dict(vane=torch.from_numpy(big.vane).pin_memory(),
              strip=torch.from_numpy(big.strip).pin_memory())
    f.find_host(hh, torch.from_numpy(big.offsets))
    b, bht = _gpu(hough, w, f=f)
    for name in oracle.CF_DTYPE.names:
        np.testing.assert_array_equal(a[name], b[name], err_msg=name)
    np.testing.assert_array_equal(aht, bht)
    f.close()
