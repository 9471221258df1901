"""The seeded synthetic inputs: the same seed gives the same windows, and
their structure is what the workloads state (detector ranges, CSR layout,
track labels, noise fraction)."""
import numpy as np

from paper_2511_02742_gb300 import synth


def test_same_seed_same_windows_other_seed_other_windows():
    a = synth.generate(50, ("poisson", 10, 1, 40), (100.0, 300.0), 0.02, seed=7)
    b = synth.generate(50, ("poisson", 10, 1, 40), (100.0, 300.0), 0.02, seed=7)
    c = synth.generate(50, ("poisson", 10, 1, 40), (100.0, 300.0), 0.02, seed=8)
    for k in ("vane", "strip", "offsets", "track", "track_offsets"):
        np.testing.assert_array_equal(getattr(a, k), getattr(b, k))
    assert not np.array_equal(a.vane, c.vane[:len(a.vane)]) or len(a.vane) != len(c.vane)
    s1 = synth.timed_stream(300, 0.6, seed=3)
    s2 = synth.timed_stream(300, 0.6, seed=3)
    np.testing.assert_array_equal(s1.t, s2.t)
    np.testing.assert_array_equal(s1.vane, s2.vane)


def test_structure_of_the_windows():
    w = synth.generate(200, ("poisson", 10, 1, 40), (100.0, 300.0), 0.05, seed=9)
    assert w.offsets[0] == 0 and (np.diff(w.offsets) >= 0).all() and w.offsets[-1] == w.n_hits
    assert ((w.vane >= 0) & (w.vane < synth.N_VANES)).all()
    assert ((w.strip >= 0) & (w.strip < synth.N_Z_STRIPS)).all()
    n_tracks = np.diff(w.track_offsets)
    assert ((n_tracks >= 1) & (n_tracks <= 40)).all()
    for k in range(w.n_windows):
        t = w.track[w.window(k)]
        assert t.max() < n_tracks[k] and t.min() >= -1
    signal = (w.track >= 0).sum()
    noise = (w.track < 0).sum()
    assert abs(noise / signal - 0.05) < 0.01
    # crossings lie inside the detector's z range, and the strip holds them
    zm = w.z_mm[w.track >= 0]
    assert (np.abs(zm) <= synth.Z_MAX_MM).all()
    strip_lo = synth.Z_MIN_MM + w.strip[w.track >= 0] * synth.Z_STRIP_PITCH_MM
    assert ((zm >= strip_lo - 1e-9) & (zm < strip_lo + synth.Z_STRIP_PITCH_MM + 1e-9)).all()


def test_stream_is_time_ordered_and_covers_the_span():
    s = synth.timed_stream(500, 0.6, noise_frac=0.02, seed=4)
    assert (np.diff(s.t) >= 0).all()
    assert s.t.min() >= 0 and s.t.max() < 500 * 1000 + 3000
    assert len(s.t) > 0.6 * 500 * 5        # some hits per decay
