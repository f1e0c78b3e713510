"""One alias table over several GPUs: two-level sampling.

The items are cut into G contiguous shards, shard g holding items
[b_g, b_{g+1}).  Each rank builds the ordinary table of its own shard (PSA,
Sec. 2.2).  A draw from the whole table picks shard g with probability
W_g / W (W_g the shard's total weight, W = sum of the W_g) and then an item of
the shard with the shard's table, so item i of shard g is drawn with
probability (W_g / W) (w_i / W_g) = w_i / W.  The only exchange between the
ranks is one allgather of the G shard totals.

A request of `count` draws is split over the shards by one multinomial draw
with p_g = W_g / W, from a generator seeded by the request's seed alone, so
every rank computes the same split without communicating.  Rank g then draws
its count_g samples from its table (the sample stream of shard g) and adds
b_g to the item indices.  The request's samples are the ranks' outputs in
shard order: grouped by shard, as the sectioned samplers of Sec. 5 group them
by section (here the sections have unequal weights).

This module is host logic only: it never touches a table's rows; the
per-shard builds and draws go through the library's C ABI on each rank.
"""
from __future__ import annotations

import numpy as np


def shard_bounds(n: int, world: int) -> list[int]:
    """b_0 .. b_G: shard g holds items [floor(g n / G), floor((g+1) n / G))."""
    if n < 0 or world < 1:
        raise ValueError("need n >= 0 and at least one shard")
    return [(g * n) // world for g in range(world + 1)]


def shard_totals(W_local: float, dist=None, device=None) -> list[float]:
    """The G shard totals W_g on every rank: one allgather of one FP64 value
    per rank through `dist` (torch.distributed with an initialised process
    group: NCCL on GPUs, gloo on CPUs); the identity without one."""
    if dist is None:
        return [float(W_local)]
    import torch
    mine = torch.tensor([float(W_local)], dtype=torch.float64, device=device)
    parts = [torch.zeros_like(mine) for _ in range(dist.get_world_size())]
    dist.all_gather(parts, mine)
    return [float(p.item()) for p in parts]


def shard_counts(count: int, seed: int, totals) -> np.ndarray:
    """How many of a request's `count` draws fall into each shard: one
    multinomial draw with p_g = W_g / W, seeded by the request's seed, so
    that every rank computes the same split.  Shards of zero weight get
    none."""
    t = np.asarray(totals, np.float64)
    if t.ndim != 1 or t.size == 0 or np.any(~np.isfinite(t)) or np.any(t < 0):
        raise ValueError("shard totals must be finite and not negative")
    W = float(t.sum())
    if W <= 0.0:
        raise ValueError("all shards have zero weight")
    if count < 0:
        raise ValueError("count must not be negative")
    rng = np.random.default_rng([int(seed) & (2**64 - 1), 0x5348])   # 'SH'
    return rng.multinomial(int(count), t / W).astype(np.int64)


def shard_offsets(counts) -> np.ndarray:
    """Start of each shard's samples in the request's output (shard order)."""
    c = np.asarray(counts, np.int64)
    out = np.zeros(c.size, np.int64)
    out[1:] = np.cumsum(c)[:-1]
    return out


def shard_stream(shard: int) -> int:
    """stream_lo of shard g's draws (stream_hi is the naive-sampling tag)."""
    return int(shard)


def to_global(local_items, shard: int, bounds) -> np.ndarray:
    """Item indices of shard `shard`'s table as indices of the whole table."""
    return np.asarray(local_items, np.int64) + int(bounds[shard])
