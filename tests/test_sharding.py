"""One table over several GPUs by two-level sampling (the sharded form of
the path): shard bounds, one allgather of the shard totals, the split of a
request's draws over the shards, and global item indices.  Two gloo
processes on the CPU stand for two GPUs; each rank's shard table is the
oracle's (test infrastructure) so that the host logic is checked without a
GPU, against the oracle on the concatenated weights:
* every item's two-level probability (W_g / W) (local mass / N_g) equals
  w_i / W (Sec. 1) within FP64 rounding;
* the draws of the two ranks, concatenated in shard order, equal a
  single-process run of the same procedure bit for bit;
* the split of the draws is identical on both ranks and sums to the count.
"""
from __future__ import annotations

import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
from paper_2106_12270_gb300 import inputs, sharding

N, COUNT, SEED = 30011, 200_003, 12


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _shard_draws(w, g, bounds, totals, count, seed):
    """Rank g's part of a request: its table (the oracle's Vose here), its
    share of the draws and their global item indices."""
    ws = w[bounds[g]: bounds[g + 1]]
    t = oracle.vose(ws)
    prob32 = t["prob"].astype(np.float32)
    c = sharding.shard_counts(count, seed, totals)
    local = oracle.sample_naive(prob32, t["alias"], 0, int(c[g]), seed,
                                sharding.shard_stream(g), 0)
    return sharding.to_global(local, g, bounds), t


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w = inputs.exponential(N, 5)
        bounds = sharding.shard_bounds(N, world)
        W_local = oracle.exact_sum(w[bounds[rank]: bounds[rank + 1]])
        totals = sharding.shard_totals(W_local, dist)
        counts = sharding.shard_counts(COUNT, SEED, totals)
        items, _ = _shard_draws(w, rank, bounds, totals, COUNT, SEED)
        dist.barrier()
        out[rank] = (totals, counts.tolist(), items.tolist())
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_two_level_table():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world, join=True,
                       start_method="spawn")
    w = inputs.exponential(N, 5)
    bounds = sharding.shard_bounds(N, world)
    totals0, counts0, _ = out[0]
    totals1, counts1, _ = out[1]
    # the allgather gave every rank the exact shard totals, in rank order
    want = [oracle.exact_sum(w[bounds[g]: bounds[g + 1]]) for g in range(world)]
    assert totals0 == totals1 == want
    # the same split of the draws on both ranks
    assert counts0 == counts1 and sum(counts0) == COUNT
    # the ranks' draws in shard order = one process doing the same
    got = np.concatenate([np.asarray(out[g][2], np.int64) for g in range(world)])
    ref = np.concatenate([_shard_draws(w, g, bounds, want, COUNT, SEED)[0]
                          for g in range(world)])
    assert np.array_equal(got, ref)
    assert np.all((got >= 0) & (got < N))
    for g in range(world):   # shard g's draws lie in shard g
        s = got[sharding.shard_offsets(counts0)[g]:][: counts0[g]]
        assert np.all((s >= bounds[g]) & (s < bounds[g + 1]))


def test_two_level_probabilities_match_the_whole_table():
    # Sec. 1: item i is drawn with probability w_i / W.  Two levels: shard g
    # with W_g / W, then item i of the shard with its table's mass / N_g.
    w = inputs.gamma(N, 9)
    W = oracle.exact_sum(w)
    for world in (1, 2, 3, 8):
        bounds = sharding.shard_bounds(N, world)
        totals = [oracle.exact_sum(w[bounds[g]: bounds[g + 1]]) for g in range(world)]
        p = np.zeros(N)
        for g in range(world):
            ws = w[bounds[g]: bounds[g + 1]]
            t = oracle.vose(ws)
            m = oracle.mass(t["prob"], t["alias"])
            p[bounds[g]: bounds[g + 1]] = (totals[g] / sum(totals)) * m / ws.size
        expect = w.astype(np.float64) / W
        assert np.max(np.abs(p - expect) / np.maximum(expect, 1.0 / N)) < 1e-9


def test_shard_split_of_the_draws():
    totals = [3.0, 0.0, 1.0]
    c = sharding.shard_counts(10**6, 7, totals)
    assert c.sum() == 10**6 and c[1] == 0
    assert abs(c[0] / 1e6 - 0.75) < 5e-3          # multinomial with p = W_g / W
    assert np.array_equal(c, sharding.shard_counts(10**6, 7, totals))   # seeded
    assert not np.array_equal(c, sharding.shard_counts(10**6, 8, totals))
    assert sharding.shard_offsets([4, 0, 6]).tolist() == [0, 4, 4]
    assert sharding.shard_bounds(10, 3) == [0, 3, 6, 10]
    assert sharding.shard_totals(2.5) == [2.5]
    with pytest.raises(ValueError):
        sharding.shard_counts(5, 1, [0.0, 0.0])
