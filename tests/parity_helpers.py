"""Shared helpers of the CUDA-vs-oracle parity tests."""
import numpy as np

import oracle
from paper_2511_02742_gb300 import synth

G = synth.GEOMETRY


def oracle_run(w, n_theta, n_rho, export=False, ids=None, geom=G, **th):
    """Oracle outputs for all windows of `w`, or for the windows `ids` only
    (each computed one by one; returned arrays indexed like `ids`)."""
    phi, z = oracle.encode(geom, w.vane, w.strip)
    if ids is None:
        return oracle.find_batch(geom, n_theta, n_rho, phi, z, w.offsets, export_acc=export, **th)
    res = []
    for k in ids:
        sl = w.window(int(k))
        r = oracle.find_window(geom, n_theta, n_rho, phi[sl], z[sl], **th)
        if not export:
            r["acc"] = None
        res.append(r)
    return res


def gpu_run(finder, w, raw=True, device="cuda", stream=None, out=None):
    import torch
    if raw:
        hits = dict(vane=torch.from_numpy(w.vane).to(device),
                    strip=torch.from_numpy(w.strip).to(device))
    else:
        phi, z = oracle.encode(finder.geometry, w.vane, w.strip)
        hits = dict(phi_q=torch.from_numpy(phi).to(device), z_q=torch.from_numpy(z).to(device))
    off = torch.from_numpy(w.offsets).to(device)
    out = finder.find(hits, off, out=out, stream=stream)
    torch.cuda.synchronize()
    return to_numpy(out, w.n_hits)


def to_numpy(out, n_hits):
    from paper_2511_02742_gb300 import hough
    r = dict(
        peaks=hough.decode_peaks(out["peaks"]),
        n_peaks=out["n_peaks"].cpu().numpy(),
        n_found=out["n_found"].cpu().numpy(),
        hit_track=out["hit_track"].cpu().numpy()[:n_hits],
        track_hits=out["track_hits"].cpu().numpy()[:n_hits],
        status=out["window_status"].cpu().numpy().astype(np.uint32),
    )
    if "acc" in out:
        r["acc"] = out["acc"].cpu().numpy()
    return r


def assert_window_equal(g, k, ref, sl, check_acc):
    """GPU batch result `g` at window k equals the oracle result `ref` (one window)."""
    n = int(ref["n_peaks"])
    assert int(g["n_peaks"][k]) == n, (k, int(g["n_peaks"][k]), n)
    assert int(g["n_found"][k]) == int(ref["n_found"]), k
    assert int(g["status"][k]) == int(ref["status"]), (k, int(g["status"][k]), int(ref["status"]))
    np.testing.assert_array_equal(g["peaks"][k][:n], ref["peaks"][:n], err_msg=f"peaks w={k}")
    np.testing.assert_array_equal(g["hit_track"][sl], ref["hit_track"], err_msg=f"hit_track w={k}")
    np.testing.assert_array_equal(g["track_hits"][sl], ref["track_hits"], err_msg=f"track_hits w={k}")
    if check_acc:
        np.testing.assert_array_equal(g["acc"][k], ref["acc"], err_msg=f"acc w={k}")


def assert_batch_equal(g, ref, w, check_acc=False):
    """Whole-batch comparison against oracle.find_batch output."""
    np.testing.assert_array_equal(g["n_peaks"], ref["n_peaks"])
    np.testing.assert_array_equal(g["n_found"], ref["n_found"])
    np.testing.assert_array_equal(g["status"], ref["status"])
    mp = ref["peaks"].shape[1]
    for k in range(w.n_windows):
        n = int(ref["n_peaks"][k])
        np.testing.assert_array_equal(g["peaks"][k][:n], ref["peaks"][k][:n],
                                      err_msg=f"peaks w={k}")
    np.testing.assert_array_equal(g["hit_track"], ref["hit_track"])
    np.testing.assert_array_equal(g["track_hits"], ref["track_hits"])
    if check_acc:
        np.testing.assert_array_equal(g["acc"], ref["acc"])
    del mp
