"""Seeded synthetic inputs shaped like the paper's workloads.

This module only draws random numbers; it holds none of the alias-table
arithmetic.  The same arrays feed the CUDA library and the CPU oracle.

The paper evaluates on uniform random weights and on shuffled power-law
weights w_i = i^-alpha in random order (Sec. 6).  The generators below cover
those and the other shapes the workloads use:

* ``uniform``           U[0,1) drawn in FP64, rounded to FP32.
* ``zipf_permuted``     w = 1/rank^s with the ranks 1..N randomly permuted.
* ``exponential``       Exp(1) drawn in FP64, rounded to FP32.
* ``gamma``             Gamma(shape, 1) in FP64, rounded to FP32 (shape 0.1
                        gives exact zeros and FP32 subnormals).
* ``log_uniform_sizes`` segment sizes floor(exp(U[ln lo, ln hi])).
* ``batched``           many segments of the above, concatenated, with
                        64-bit offsets.

The elementwise draws (uniform, exponential, gamma) come in chunks of 2^24
items: chunk k is drawn in FP64 by ``numpy.random.default_rng([seed, k])``
and rounded to FP32, so every chunk is its own seeded stream and the chunks
are filled by a pool of host threads (numpy releases the GIL while it
draws).  The permutation of ``zipf_permuted`` comes from one
``default_rng(seed)`` stream.
"""
from __future__ import annotations

import concurrent.futures as cf
import math
import os

import numpy as np

_CHUNK = 1 << 24


def _chunked(n: int, seed: int, draw) -> np.ndarray:
    """out[k*2^24 : (k+1)*2^24] = draw(default_rng([seed, k]), size) as FP32."""
    out = np.empty(n, np.float32)

    def fill(k):
        a = k * _CHUNK
        b = min(n, a + _CHUNK)
        out[a:b] = draw(np.random.default_rng([seed, k]), b - a).astype(np.float32)

    nchunks = (n + _CHUNK - 1) // _CHUNK
    if nchunks <= 1:
        for k in range(nchunks):
            fill(k)
    else:
        with cf.ThreadPoolExecutor(max_workers=min(nchunks, os.cpu_count() or 1)) as ex:
            list(ex.map(fill, range(nchunks)))
    return out


def uniform(n: int, seed: int) -> np.ndarray:
    return _chunked(n, seed, lambda rng, m: rng.random(m))


def zipf_permuted(n: int, seed: int, s: float = 1.0) -> np.ndarray:
    rng = np.random.default_rng(seed)
    rank = rng.permutation(n).astype(np.float64) + 1.0
    out = np.empty(n, np.float32)
    for a in range(0, n, _CHUNK):
        b = min(n, a + _CHUNK)
        out[a:b] = (1.0 / np.power(rank[a:b], s)).astype(np.float32)
    return out


def exponential(n: int, seed: int) -> np.ndarray:
    return _chunked(n, seed, lambda rng, m: rng.exponential(1.0, m))


def gamma(n: int, seed: int, shape: float = 0.1) -> np.ndarray:
    return _chunked(n, seed, lambda rng, m: rng.gamma(shape, 1.0, m))


def log_uniform_sizes(count: int, seed: int, lo: int, hi: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    x = np.floor(np.exp(rng.uniform(math.log(lo), math.log(hi), count)))
    return np.clip(x, lo, hi).astype(np.int64)


def batched(sizes, seed: int, kind: str = "gamma", **kw):
    """Concatenate one segment per size; returns (weights f32, offsets u64)."""
    sizes = np.asarray(sizes, np.int64)
    off = np.zeros(sizes.size + 1, np.uint64)
    off[1:] = np.cumsum(sizes).astype(np.uint64)
    total = int(off[-1])
    gen = {"gamma": gamma, "uniform": uniform, "exponential": exponential}[kind]
    return gen(total, seed, **kw), off


def by_name(kind: str, n: int, seed: int) -> np.ndarray:
    """Named weight distributions used by tests and the benchmark."""
    if kind == "uniform":
        return uniform(n, seed)
    if kind == "zipf":
        return zipf_permuted(n, seed, 1.0)
    if kind == "zipf0.5":
        return zipf_permuted(n, seed, 0.5)
    if kind == "exponential":
        return exponential(n, seed)
    if kind == "gamma":
        return gamma(n, seed, 0.1)
    raise ValueError(kind)


def serving_stream(nreq: int, seed: int, rate_per_s: float, build_range=(1_000, 10_000_000),
                   sample_range=(100, 1_000_000), mix=(0.10, 0.85, 0.05)):
    """Poisson request stream: list of dicts with arrival time `t` (s) and
    `op` in {"build", "sample", "release"}; builds carry a size (log-uniform
    in build_range) and a weight kind ("uniform" or "zipf", 50/50), samples a
    draw count (log-uniform in sample_range), a seed and the index of the
    earlier build they draw from, releases the index of a build.  The first
    request is always a build.  Which tables exist at a sample is decided by
    the stream itself (a sample never names a released table)."""
    rng = np.random.default_rng(seed)
    t = 0.0
    ops = []
    live = []
    for k in range(nreq):
        t += rng.exponential(1.0 / rate_per_s)
        u = rng.random()
        if not live or u < mix[0]:
            n = int(np.floor(np.exp(rng.uniform(math.log(build_range[0]),
                                                 math.log(build_range[1])))))
            ops.append({"t": t, "op": "build", "n": n,
                        "kind": "uniform" if rng.random() < 0.5 else "zipf",
                        "wseed": int(rng.integers(1, 2**31))})
            live.append(len(ops) - 1)
        elif u < mix[0] + mix[1]:
            c = int(np.floor(np.exp(rng.uniform(math.log(sample_range[0]),
                                                math.log(sample_range[1])))))
            src = live[int(rng.integers(0, len(live)))]
            ops.append({"t": t, "op": "sample", "count": c, "table": src,
                        "seed": int(rng.integers(0, 2**63)), "stream": k})
        else:
            src = live.pop(int(rng.integers(0, len(live))))
            ops.append({"t": t, "op": "release", "table": src})
    return ops
