"""Host-side sharding of a window batch over replicas (one process per GPU).

Windows are independent units of work (one CTA per window on the device), so
a batch is split into contiguous window ranges with about the same number of
hits each; every rank runs its range on its own GPU and the per-window
results are concatenated in window order on the host.  No collective touches
the data path; torch.distributed is used only to move finished results.
"""
from __future__ import annotations

import numpy as np


def shard_ranges(offsets, world_size: int):
    """Contiguous [begin, end) window ranges, one per rank, balanced by hits.

    Boundaries are placed where the running hit count crosses k/world_size of
    the total; every window belongs to exactly one range, ranges are in order,
    and an empty batch gives empty ranges."""
    offsets = np.asarray(offsets, dtype=np.int64)
    n_windows = len(offsets) - 1
    if world_size < 1:
        raise ValueError("world_size must be >= 1")
    total = int(offsets[-1] - offsets[0]) if n_windows > 0 else 0
    bounds = [0]
    for k in range(1, world_size):
        target = offsets[0] + (total * k) // world_size
        # first window whose start is >= target, not before the previous bound
        b = int(np.searchsorted(offsets[:-1], target, side="left")) if n_windows > 0 else 0
        bounds.append(max(bounds[-1], min(b, n_windows)))
    bounds.append(n_windows)
    return [(bounds[k], bounds[k + 1]) for k in range(world_size)]


def local_windows(w, rank: int, world_size: int):
    """The rank's slice of a synth.Windows batch (hits re-based to 0)."""
    from .synth import Windows
    b, e = shard_ranges(w.offsets, world_size)[rank]
    h0, h1 = int(w.offsets[b]), int(w.offsets[e])
    t0, t1 = int(w.track_offsets[b]), int(w.track_offsets[e])
    return Windows(w.vane[h0:h1], w.strip[h0:h1], w.offsets[b:e + 1] - h0, w.track[h0:h1],
                   w.z_mm[h0:h1], w.track_params[t0:t1], w.track_offsets[b:e + 1] - t0)


def concat_results(parts):
    """Concatenate per-rank result dicts (window-major arrays and hit arrays) in rank order."""
    keys = parts[0].keys()
    return {k: np.concatenate([p[k] for p in parts]) for k in keys if parts[0][k] is not None}
