"""Multi-replica path on CPU: world-size-2 gloo ranks shard the windows,
compute their range (the oracle stands in for the GPU here) and rank 0
concatenates the results in window order; they must equal a single-process run."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2511_02742_gb300 import shard, synth


def test_shard_ranges_partition_and_balance():
    rng = np.random.default_rng(0)
    for world in (1, 2, 3, 8):
        lens = rng.integers(0, 50, 1000)
        off = np.zeros(1001, np.int64)
        off[1:] = np.cumsum(lens)
        r = shard.shard_ranges(off, world)
        assert r[0][0] == 0 and r[-1][1] == 1000
        for (a, b), (c, d) in zip(r, r[1:]):
            assert b == c and a <= b
        hits = [off[b] - off[a] for a, b in r]
        assert max(hits) - min(hits) <= 2 * lens.max()
    assert shard.shard_ranges(np.zeros(1, np.int64), 4) == [(0, 0)] * 4
    one = shard.shard_ranges(np.array([0, 10], np.int64), 3)
    assert sum(b - a for a, b in one) == 1


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    w = synth.generate(64, ("poisson", 6, 1, 20), (100.0, 300.0), 0.02, seed=21)
    lw = shard.local_windows(w, rank, world)
    phi, z = oracle.encode(synth.GEOMETRY, lw.vane, lw.strip)
    r = oracle.find_batch(synth.GEOMETRY, 128, 128, phi, z, lw.offsets)
    r["peaks"] = r["peaks"].reshape(-1)
    parts = [None] * world
    dist.all_gather_object(parts, r)
    if rank == 0:
        q.put(shard.concat_results(parts))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_gloo_sharding_equals_single_process():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    import oracle
    w = synth.generate(64, ("poisson", 6, 1, 20), (100.0, 300.0), 0.02, seed=21)
    phi, z = oracle.encode(synth.GEOMETRY, w.vane, w.strip)
    ref = oracle.find_batch(synth.GEOMETRY, 128, 128, phi, z, w.offsets)
    for k in ("n_peaks", "n_found", "hit_track", "track_hits", "status"):
        np.testing.assert_array_equal(got[k], ref[k], err_msg=k)
    np.testing.assert_array_equal(got["peaks"], ref["peaks"].reshape(-1))
