"""Seeded synthetic detector input for the track-finding path.

This module is the stand-in for the paper's Geant4 -> EventPileup -> StripDigi
chain (Section 3), which is not available here.  It produces strip-level hits
(vane index, z-strip index) grouped into time windows, plus generator truth.
It contains none of the track-finding arithmetic (no Hough transform, no
binning, no peak or association logic): both the CUDA path and the CPU oracle
consume its output, and each encodes and processes it with its own code.

Physics model:
  * detector geometry of Section 2: 40 radial vanes, z sensitive range
    +-194.56 mm (4 Z-sensors x 512 strips at 0.19 mm), radial sensitive range
    70-290 mm split into two R-sensor rows [70, 167.28] and [192.72, 290];
  * 300 MeV/c muons on a circular orbit r = 333 mm, z = 0 in a uniform 3 T
    field along z (Sections 2 and 3);
  * decay positron: momentum p ~ U[p_lo, p_hi] MeV/c, direction = the muon's
    tangent rotated in-plane by alpha ~ U(-30, 30) deg, dip lambda ~
    U(-15, 15) deg; an ideal helix (no energy loss, no scattering),
    transverse radius R = p_T / (0.3 B) (p_T in GeV/c, R in m);
  * a hit is every crossing of the helix with a vane half-plane inside an
    R-sensor row and inside |z| <= 194.56 mm, within the first turn (or the
    first `max_turns` turns); its z is digitised to the strip that contains it;
  * noise: round(nu * n_signal) hits per window at a uniform vane and strip;
  * the hits of a window are shuffled so that tracks interleave.

Random numbers come from numpy's PCG64 Generator seeded explicitly.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

# ---- detector constants (Section 2) -------------------------------------
N_VANES = 40
VANE_PITCH_DEG = 360.0 / N_VANES          # 9 degrees between radial vanes
Z_STRIP_PITCH_MM = 0.19                   # 190 um strip pitch
N_Z_STRIPS = 4 * 512                      # 4 Z-sensors along z, 512 strips each
Z_MIN_MM = -0.5 * N_Z_STRIPS * Z_STRIP_PITCH_MM   # -194.56 mm
Z_MAX_MM = -Z_MIN_MM
R_SENSOR_ROWS_MM = ((70.0, 70.0 + 97.28), (290.0 - 97.28, 290.0))
B_FIELD_T = 3.0
MUON_ORBIT_R_MM = 333.0

# Fixed-point geometry handed to the library and to the oracle: 1 unit is
# 1/200 of a degree in phi and 1/200 of a millimetre in z, so the strip pitch
# of 0.19 mm is exactly 38 units and a vane step of 9 degrees is 1800 units.
GEOMETRY = dict(
    n_vanes=N_VANES,
    n_z_strips=N_Z_STRIPS,
    z_pitch_u=38,
    z_min_u=-38912,
    phi_u_per_deg=200,
    z_u_per_mm=200,
    rho_min=-500.0,
    rho_max=500.0,
)


@dataclass
class Windows:
    """A batch of time windows in CSR form.

    vane, strip : int32[H]   strip address of each RecoHit
    offsets     : int64[W+1] window w owns hits offsets[w]:offsets[w+1]
    track       : int32[H]   generator track id within its window, -1 = noise
    z_mm        : float64[H] undigitised crossing z (nan for noise)
    track_params: float64[n_tracks, 4] (p, alpha_deg, lambda_deg, phi_mu_deg)
    track_offsets: int64[W+1] window w owns tracks track_offsets[w]:...[w+1]
    """
    vane: np.ndarray
    strip: np.ndarray
    offsets: np.ndarray
    track: np.ndarray
    z_mm: np.ndarray
    track_params: np.ndarray
    track_offsets: np.ndarray

    @property
    def n_windows(self) -> int:
        return len(self.offsets) - 1

    @property
    def n_hits(self) -> int:
        return int(self.offsets[-1])

    def window(self, w: int) -> slice:
        return slice(int(self.offsets[w]), int(self.offsets[w + 1]))

    def subset(self, ids) -> "Windows":
        """A new batch holding windows `ids` (in that order)."""
        ids = np.asarray(ids, dtype=np.int64)
        lens = self.offsets[ids + 1] - self.offsets[ids]
        idx = np.concatenate([np.arange(self.offsets[i], self.offsets[i + 1]) for i in ids]) \
            if len(ids) else np.zeros(0, np.int64)
        tl = self.track_offsets[ids + 1] - self.track_offsets[ids]
        tidx = np.concatenate([np.arange(self.track_offsets[i], self.track_offsets[i + 1]) for i in ids]) \
            if len(ids) else np.zeros(0, np.int64)
        off = np.zeros(len(ids) + 1, np.int64)
        np.cumsum(lens, out=off[1:])
        toff = np.zeros(len(ids) + 1, np.int64)
        np.cumsum(tl, out=toff[1:])
        return Windows(self.vane[idx], self.strip[idx], off, self.track[idx], self.z_mm[idx],
                       self.track_params[tidx], toff)


def _helix_crossings(p, alpha, lam, phi_mu, max_turns=1):
    """Vane crossings of ideal positron helices.

    All angles in radians.  Returns (vane[N, 40, 2*T], z[...], ok[...], s[...]) for T =
    max_turns, where s is the transverse arc length (mm) from the decay point.
    """
    n = p.shape[0]
    p_t = p * np.cos(lam)
    radius = p_t / (0.3 * B_FIELD_T)          # mm when p_t in MeV/c
    x0 = MUON_ORBIT_R_MM * np.cos(phi_mu)
    y0 = MUON_ORBIT_R_MM * np.sin(phi_mu)
    # A positive particle in B along +z turns clockwise seen from +z; the muon's
    # velocity at azimuth phi is (sin phi, -cos phi).  Rotate it by alpha.
    ux = np.sin(phi_mu) * np.cos(alpha) - (-np.cos(phi_mu)) * np.sin(alpha)
    uy = np.sin(phi_mu) * np.sin(alpha) + (-np.cos(phi_mu)) * np.cos(alpha)
    # Centre of curvature lies to the right of the velocity for clockwise motion.
    xc = x0 + radius * uy
    yc = y0 - radius * ux
    psi0 = np.arctan2(y0 - yc, x0 - xc)

    vane_ang = np.deg2rad(np.arange(N_VANES) * VANE_PITCH_DEG)       # (40,)
    cv = np.cos(vane_ang)[None, :]
    sv = np.sin(vane_ang)[None, :]
    d = sv * xc[:, None] - cv * yc[:, None]                           # (N, 40)
    ratio = d / radius[:, None]
    has = np.abs(ratio) < 1.0
    a = np.arcsin(np.clip(ratio, -1.0, 1.0))
    psi = np.stack([vane_ang[None, :] + a, vane_ang[None, :] + math.pi - a], axis=-1)  # (N,40,2)
    # Clockwise: psi decreases with arc length.
    dpsi = np.mod(psi0[:, None, None] - psi, 2.0 * math.pi)
    dpsi = np.concatenate([dpsi + 2.0 * math.pi * m for m in range(max_turns)], axis=-1)
    psi = np.concatenate([psi] * max_turns, axis=-1)
    has = has[..., None]
    s = radius[:, None, None] * dpsi
    x = xc[:, None, None] + radius[:, None, None] * np.cos(psi)
    y = yc[:, None, None] + radius[:, None, None] * np.sin(psi)
    r_along = x * cv[..., None] + y * sv[..., None]                  # signed radius on the vane
    z = s * np.tan(lam)[:, None, None]
    in_row = np.zeros(psi.shape, dtype=bool)
    for lo, hi in R_SENSOR_ROWS_MM:
        in_row |= (r_along >= lo) & (r_along <= hi)
    ok = has & in_row & (np.abs(z) <= Z_MAX_MM) & (s > 0.0)
    vane = np.broadcast_to(np.arange(N_VANES, dtype=np.int32)[None, :, None], ok.shape)
    return vane, z, ok, s


def _digitise_z(z_mm):
    """Strip containing z (StripDigi stand-in); clipped to the sensor."""
    j = np.floor((z_mm - Z_MIN_MM) / Z_STRIP_PITCH_MM).astype(np.int64)
    return np.clip(j, 0, N_Z_STRIPS - 1).astype(np.int32)


def _tracks_per_window(rng, n_windows, tracks):
    if isinstance(tracks, (int, np.integer)):
        return np.full(n_windows, int(tracks), dtype=np.int64)
    kind = tracks[0]
    if kind == "poisson":
        _, mean, lo, hi = tracks
        return np.clip(rng.poisson(mean, n_windows), lo, hi).astype(np.int64)
    if kind == "uniform":
        _, lo, hi = tracks
        return rng.integers(lo, hi + 1, n_windows).astype(np.int64)
    raise ValueError(f"unknown track-count law {tracks!r}")


def generate(n_windows: int, tracks, p_range=(100.0, 300.0), noise_frac=0.0, seed=0,
             shuffle=True, alpha_deg=30.0, lambda_deg=15.0, max_turns=1) -> Windows:
    """Generate `n_windows` pileup windows.

    tracks: an int (fixed count per window), ("poisson", mean, lo, hi) or
    ("uniform", lo, hi).  max_turns: how many transverse turns of each helix
    may leave hits (the track still ends when it leaves |z| <= 194.56 mm).
    """
    rng = np.random.default_rng(seed)
    ntr = _tracks_per_window(rng, n_windows, tracks)
    n_tracks = int(ntr.sum())
    p = rng.uniform(p_range[0], p_range[1], n_tracks)
    alpha = np.deg2rad(rng.uniform(-alpha_deg, alpha_deg, n_tracks))
    lam = np.deg2rad(rng.uniform(-lambda_deg, lambda_deg, n_tracks))
    phi_mu = rng.uniform(0.0, 2.0 * math.pi, n_tracks)

    vane_all = []
    z_all = []
    trk_all = []
    chunk = 1 << 16
    for c0 in range(0, n_tracks, chunk):
        c1 = min(n_tracks, c0 + chunk)
        vane, z, ok, _ = _helix_crossings(p[c0:c1], alpha[c0:c1], lam[c0:c1], phi_mu[c0:c1],
                                          max_turns)
        ti, vi, si = np.nonzero(ok)
        vane_all.append(vane[ti, vi, si])
        z_all.append(z[ti, vi, si])
        trk_all.append(ti.astype(np.int64) + c0)
    vane_sig = np.concatenate(vane_all) if vane_all else np.zeros(0, np.int32)
    z_sig = np.concatenate(z_all) if z_all else np.zeros(0)
    trk_global = np.concatenate(trk_all) if trk_all else np.zeros(0, np.int64)

    track_off = np.zeros(n_windows + 1, np.int64)
    np.cumsum(ntr, out=track_off[1:])
    win_of_track = np.repeat(np.arange(n_windows, dtype=np.int64), ntr)
    sig_win = win_of_track[trk_global]
    sig_local = (trk_global - track_off[sig_win]).astype(np.int32)
    n_sig = np.bincount(sig_win, minlength=n_windows)
    n_noise = np.rint(noise_frac * n_sig).astype(np.int64)
    tot_noise = int(n_noise.sum())
    noise_win = np.repeat(np.arange(n_windows, dtype=np.int64), n_noise)
    noise_vane = rng.integers(0, N_VANES, tot_noise).astype(np.int32)
    noise_strip = rng.integers(0, N_Z_STRIPS, tot_noise).astype(np.int32)

    win = np.concatenate([sig_win, noise_win])
    vane_h = np.concatenate([vane_sig.astype(np.int32), noise_vane])
    strip_h = np.concatenate([_digitise_z(z_sig), noise_strip])
    trk_h = np.concatenate([sig_local, np.full(tot_noise, -1, np.int32)])
    z_h = np.concatenate([z_sig, np.full(tot_noise, np.nan)])
    key = rng.random(len(win)) if shuffle else np.arange(len(win), dtype=np.float64)
    order = np.lexsort((key, win))
    counts = np.bincount(win, minlength=n_windows)
    off = np.zeros(n_windows + 1, np.int64)
    np.cumsum(counts, out=off[1:])
    params = np.stack([p, np.rad2deg(alpha), np.rad2deg(lam), np.rad2deg(phi_mu)], axis=1)
    return Windows(vane_h[order].copy(), strip_h[order].copy(), off, trk_h[order].copy(),
                   z_h[order].copy(), params, track_off)


@dataclass
class TimedHits:
    """A time-ordered hit stream (Section 5 time slicing): t in picoseconds."""
    t: np.ndarray          # int64 [n], non-decreasing
    vane: np.ndarray       # int32 [n]
    strip: np.ndarray      # int32 [n]
    track: np.ndarray      # int64 [n]: generating track, -1 for noise

    @property
    def n_hits(self) -> int:
        return len(self.t)


def timed_stream(duration_ns: float, rate_per_ns: float, p_range=(100.0, 300.0),
                 noise_frac=0.0, seed=0, spread_ps=2000) -> TimedHits:
    """Decays as a Poisson process of `rate_per_ns` over `duration_ns` (the
    paper's pileup rates are 0.06, 0.6 and 6 decays per ns); each track's
    hits arrive within `spread_ps` of its decay time; noise hits are spread
    uniformly over the stream.  Hits are sorted by time (stable)."""
    rng = np.random.default_rng(seed)
    dur_ps = int(round(duration_ns * 1000))
    n_tracks = int(rng.poisson(rate_per_ns * duration_ns))
    w = generate(n_tracks, 1, p_range, 0.0, seed=int(rng.integers(1 << 31)), shuffle=False)
    t_dec = rng.integers(0, max(dur_ps, 1), n_tracks)
    trk = np.repeat(np.arange(n_tracks, dtype=np.int64), np.diff(w.offsets))
    t_sig = t_dec[trk] + rng.integers(0, spread_ps, len(trk))
    n_noise = int(round(noise_frac * len(trk)))
    t_noise = rng.integers(0, max(dur_ps, 1) + spread_ps, n_noise)
    t = np.concatenate([t_sig, t_noise]).astype(np.int64)
    vane = np.concatenate([w.vane, rng.integers(0, N_VANES, n_noise).astype(np.int32)])
    strip = np.concatenate([w.strip, rng.integers(0, N_Z_STRIPS, n_noise).astype(np.int32)])
    track = np.concatenate([trk, np.full(n_noise, -1, np.int64)])
    order = np.argsort(t, kind="stable")
    return TimedHits(t[order].copy(), vane[order].copy(), strip[order].copy(), track[order].copy())


def line_window(theta_deg: float, rho: float, vanes=None) -> Windows:
    """One window whose hits lie on the straight line phi*cos(theta) + z*sin(theta) = rho
    (phi in degrees at each vane, z in mm), digitised to strips; vanes whose
    crossing leaves the z range are skipped.  Used for closed-form checks."""
    th = math.radians(theta_deg)
    vanes = range(N_VANES) if vanes is None else vanes
    vv, ss, zz = [], [], []
    for k in vanes:
        phi = k * VANE_PITCH_DEG
        if abs(math.sin(th)) < 1e-12:
            continue
        z = (rho - phi * math.cos(th)) / math.sin(th)
        if abs(z) >= Z_MAX_MM:
            continue
        vv.append(k)
        zz.append(z)
        ss.append(int(_digitise_z(np.array([z]))[0]))
    n = len(vv)
    return Windows(np.array(vv, np.int32), np.array(ss, np.int32), np.array([0, n], np.int64),
                   np.zeros(n, np.int32), np.array(zz), np.zeros((1, 4)), np.array([0, 1], np.int64))


def concat(parts) -> Windows:
    """Concatenate batches window-wise."""
    offs = [np.zeros(1, np.int64)]
    toffs = [np.zeros(1, np.int64)]
    base = 0
    tbase = 0
    for w in parts:
        offs.append(w.offsets[1:] + base)
        toffs.append(w.track_offsets[1:] + tbase)
        base += w.n_hits
        tbase += int(w.track_offsets[-1])
    return Windows(np.concatenate([w.vane for w in parts]).astype(np.int32),
                   np.concatenate([w.strip for w in parts]).astype(np.int32),
                   np.concatenate(offs), np.concatenate([w.track for w in parts]).astype(np.int32),
                   np.concatenate([w.z_mm for w in parts]),
                   np.concatenate([w.track_params for w in parts]), np.concatenate(toffs))


# ---- named workloads (shapes and distributions of the paper's pileup) ----
WORKLOADS = {
    # 10 windows x 1 track, 256x256 accumulator
    "tiny": dict(n_windows=10, tracks=1, p_range=(100.0, 300.0), noise_frac=0.0,
                 n_theta=256, n_rho=256, seed=0),
    # 1000 windows x 5 tracks, 1% noise, 512x512
    "plain": dict(n_windows=1000, tracks=5, p_range=(100.0, 300.0), noise_frac=0.01,
                  n_theta=512, n_rho=512, seed=0),
    # 1e5 windows, Poisson(10) tracks clipped to [1, 40], 2% noise, 512x512
    "batched": dict(n_windows=100000, tracks=("poisson", 10, 1, 40), p_range=(100.0, 300.0),
                    noise_frac=0.02, n_theta=512, n_rho=512, seed=0),
    # 1e4 windows x 40 tracks, p in [50, 300], 5% noise, 1024x1024.  Hits may
    # come from up to 4 transverse turns so that a window holds ~1e3 hits.
    "high_pileup": dict(n_windows=10000, tracks=40, p_range=(50.0, 300.0), noise_frac=0.05,
                        n_theta=1024, n_rho=1024, seed=0, max_turns=4),
    # serving: windows of 1-40 tracks arriving as a Poisson stream, 512x512
    "serving": dict(n_windows=None, tracks=("uniform", 1, 40), p_range=(100.0, 300.0),
                    noise_frac=0.02, n_theta=512, n_rho=512, seed=0, rate_windows_per_s=1e5),
}


def workload(name: str, n_windows: int | None = None, seed: int | None = None) -> Windows:
    cfg = WORKLOADS[name]
    nw = n_windows if n_windows is not None else cfg["n_windows"]
    return generate(nw, cfg["tracks"], cfg["p_range"], cfg["noise_frac"],
                    cfg["seed"] if seed is None else seed, max_turns=cfg.get("max_turns", 1))
