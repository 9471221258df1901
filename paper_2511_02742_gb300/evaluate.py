"""Track-finding efficiency against generator truth (Section 7, Eq. (2)).

epsilon = N_found / N_all: a generated track counts as found when one
extended track holds hits of it on at least `min_run` consecutive vanes
(five in Section 7; the vanes form a ring, so runs wrap around).  This is
host-side analysis of the library's outputs and the generator's labels; it
takes no part in finding tracks.
"""
from __future__ import annotations

import numpy as np


def _has_run(vanes: np.ndarray, n_vanes: int, min_run: int) -> bool:
    """Whether the set of vanes holds min_run consecutive ones (mod n_vanes)."""
    on = np.zeros(n_vanes, bool)
    on[np.asarray(vanes, np.int64) % n_vanes] = True
    if on.all():
        return min_run <= n_vanes
    start = int(np.flatnonzero(~on)[0])          # walk the ring from an empty vane
    run = best = 0
    for k in range(1, n_vanes + 1):
        if on[(start + k) % n_vanes]:
            run += 1
            best = max(best, run)
        else:
            run = 0
    return best >= min_run


def efficiency(vane, truth, offsets, track_offsets, ext_track, n_vanes: int = 40,
               min_run: int = 5) -> dict:
    """epsilon over a batch: vane, truth (generator track id within its window,
    -1 noise), offsets (CSR windows), track_offsets (generated tracks per
    window), ext_track (window-local extended-track index per hit, -1 none).

    Returns dict(found, all, epsilon, findable, epsilon_findable): `findable`
    counts generated tracks whose own hits have such a run at all."""
    vane = np.asarray(vane)
    truth = np.asarray(truth)
    ext_track = np.asarray(ext_track)
    offsets = np.asarray(offsets, np.int64)
    track_offsets = np.asarray(track_offsets, np.int64)
    found = findable = 0
    n_all = int(track_offsets[-1] - track_offsets[0])
    for w in range(len(offsets) - 1):
        s = slice(int(offsets[w]), int(offsets[w + 1]))
        v, t, x = vane[s], truth[s], ext_track[s]
        for g in range(int(track_offsets[w + 1] - track_offsets[w])):
            mine = t == g
            if not mine.any() or not _has_run(v[mine], n_vanes, min_run):
                continue
            findable += 1
            for tr in np.unique(x[mine & (x >= 0)]):
                if _has_run(v[mine & (x == tr)], n_vanes, min_run):
                    found += 1
                    break
    return dict(found=found, all=n_all, epsilon=found / n_all if n_all else 0.0,
                findable=findable, epsilon_findable=found / findable if findable else 0.0)
