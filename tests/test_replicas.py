"""The multi-GPU form of the path is replicas (independent tables per rank,
no data-path collective).  Its host logic -- environment, per-rank seeds,
max-over-ranks timing, job throughput -- runs here as two gloo processes on
the CPU (no GPU)."""
from __future__ import annotations

import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2106_12270_gb300 import inputs, replicas


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, wsz, loc = replicas.env()
        seed = replicas.rank_seed(3, r)
        w = inputs.by_name("zipf", 1000, seed)
        # each rank "measures" its own times; the job keeps the slowest
        times = [10.0 + r, 5.0 - r, float(w[0])]
        mx = replicas.max_over_ranks(times, dist)
        dist.barrier()
        out[r] = (r, wsz, loc, seed, float(w[:10].sum()), mx)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_replicas():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world, join=True,
                       start_method="spawn")
    res = [out[r] for r in range(world)]
    # environment read back per rank
    assert [(r[0], r[1], r[2]) for r in res] == [(0, 2, 0), (1, 2, 1)]
    # independent tables: different seeds and different weights
    assert res[0][3] != res[1][3] and res[0][4] != res[1][4]
    # every rank sees the element-wise maximum of all ranks' times
    assert res[0][5] == res[1][5]
    assert res[0][5][0] == 11.0 and res[0][5][1] == 5.0
    assert res[0][5][2] == max(inputs.by_name("zipf", 1000, 3)[0], inputs.by_name("zipf", 1000, 4)[0])


def test_single_process_is_identity_and_job_rate():
    assert replicas.max_over_ranks([1.5, 2.5]) == [1.5, 2.5]
    # weak scaling: 4 ranks, 1e8 items each, slowest rank 2 ms -> 2e11 items/s
    assert replicas.job_rate(1e8, 4, 2.0) == pytest.approx(2e11)
    assert replicas.rank_seed(3, 0) != replicas.rank_seed(3, 1)
