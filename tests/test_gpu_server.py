"""The request loop (continuous batching over resident tables), GPU.

Every result must be the same alone and in the mix: a served table equals a
single build of the same weights bit for bit, and a served sample equals
wrs_sample_rows on that table (and the oracle's sampler) bit for bit.
Admission by HBM budget, unknown/released tables and data errors are
checked through request statuses.
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle
import paper_2106_12270_gb300 as wrs
from gpu_util import Built, gpu_sample
from paper_2106_12270_gb300 import inputs, serving

pytestmark = pytest.mark.gpu


def served_rows(srv, ticket, n):
    dst = torch.empty(n, dtype=torch.int64)
    srv.export(ticket, dst)
    return dst


def test_served_equals_alone():
    srv = wrs.Server(2 << 30, 3)
    try:
        sizes = [1, 17, 1000, 4097, 65536, 300_001]
        ws, tks = [], []
        for k, n in enumerate(sizes):
            w = inputs.by_name(["uniform", "zipf", "gamma"][k % 3], n, 40 + k)
            if w.sum() == 0:
                w[0] = 1.0
            t = torch.from_numpy(w)
            t = t.cuda() if k % 2 else t.pin_memory()
            ws.append(w)
            tks.append(srv.build(t))
        outs = []
        for k, tk in enumerate(tks):
            for j, count in enumerate((1, 1000, 123_457)):
                dev = (k + j) % 2 == 0
                out = torch.empty(count, dtype=torch.int32, device="cuda" if dev else "cpu")
                if not dev:
                    out = out.pin_memory()
                outs.append((k, count, 1000 * k + j, srv.sample(tk, count, 77 + j, out, 1000 * k + j), out))
        for tk in tks:
            assert srv.wait(tk) == wrs.OK
        for k, count, slo, tk, out in outs:
            assert srv.wait(tk) == wrs.OK
        for k, (w, tk) in enumerate(zip(ws, tks)):
            alone = Built(w)
            rows = served_rows(srv, tk, w.size)
            assert torch.equal(rows, alone.rows_t.cpu()), k
        for k, count, slo, tk, out in outs:
            alone = Built(ws[k])
            want = gpu_sample(alone.rows_t, ws[k].size, 0, count, 77 + (slo % 1000), slo, 0)
            got = out.cpu().numpy().view(np.uint32)
            assert np.array_equal(got, want), (k, count)
        st = srv.stats()
        assert st["completed"] == len(tks) + len(outs) and st["errors"] == 0
    finally:
        srv.close()


def test_poisson_mix_same_as_alone():
    ops = inputs.serving_stream(400, 5, 4000.0, build_range=(1_000, 200_000),
                                sample_range=(100, 100_000))
    srv = wrs.Server(4 << 30, 4)
    try:
        tickets, outputs, weights, status = serving.replay(srv, ops)
        assert all(s == wrs.OK for s in status.values())
        st = srv.stats()
        assert st["completed"] == len(ops)
        assert 0 < st["p50_ms"] <= st["p99_ms"]
        assert st["steps"] < len(ops)   # requests were batched
        # every 10th sample: identical to drawing from a lone build
        checked = 0
        for k, op in enumerate(ops):
            if op["op"] != "sample" or k % 10:
                continue
            src = op["table"]
            w = weights[src].cpu().numpy()
            alone = Built(w)
            want = gpu_sample(alone.rows_t, w.size, 0, op["count"], op["seed"], op["stream"], 0)
            assert np.array_equal(outputs[k][: op["count"]].cpu().numpy().view(np.uint32), want)
            # and the oracle's sampler on that table
            o = oracle.sample_naive(alone.prob, alone.alias, 0, min(op["count"], 5000),
                                    op["seed"], op["stream"], 0)
            assert np.array_equal(want[: o.size], o)
            checked += 1
        assert checked > 5
    finally:
        srv.close()


def test_admission_by_budget():
    n = 100_000                    # 0.8 MB resident, ~1.2 MB while building
    srv = wrs.Server(3_000_000, 2)
    try:
        w = [torch.from_numpy(inputs.uniform(n, s)).cuda() for s in range(3)]
        t0 = srv.build(w[0])
        t1 = srv.build(w[1])
        assert srv.wait(t0) == wrs.OK and srv.wait(t1) == wrs.OK
        t2 = srv.build(w[2])           # needs a release first: 1.6 + 2.0 MB > 3 MB
        import time
        time.sleep(0.2)
        assert srv.poll(t2) == (False, wrs.OK)
        r = srv.release(t0)
        assert srv.wait(r) == wrs.OK
        assert srv.wait(t2) == wrs.OK
        big = torch.ones(1_000_000, device="cuda")
        assert srv.wait(srv.build(big)) == wrs.ENOMEM   # can never fit
        st = srv.stats()
        assert st["peak_bytes"] <= 3_000_000
    finally:
        srv.close()


def test_unknown_released_and_bad_tables():
    srv = wrs.Server(1 << 30, 2)
    try:
        out = torch.empty(10, dtype=torch.int32, device="cuda")
        assert srv.wait(srv.sample(987654321, 10, 1, out)) == wrs.ENOTFOUND
        w = torch.from_numpy(inputs.uniform(1000, 3)).cuda()
        t = srv.build(w)
        assert srv.wait(srv.release(t)) == wrs.OK
        assert srv.wait(srv.sample(t, 10, 1, out)) == wrs.ENOTFOUND
        bad = torch.from_numpy(inputs.uniform(1000, 4)).cuda()
        bad[10] = float("nan")
        tb = srv.build(bad)
        s = srv.sample(tb, 10, 1, out)
        assert srv.wait(tb) == wrs.ENONFINITE
        assert srv.wait(s) == wrs.ENONFINITE
        z = torch.zeros(50, device="cuda")
        assert srv.wait(srv.build(z)) == wrs.EZEROSUM
    finally:
        srv.close()


def test_large_builds_single_table_path():
    """Tables of 2^17 items and more take the multi-CTA pipeline: the same
    rows as a single build, data errors reported per table, memory given
    back on release."""
    srv = wrs.Server(1 << 30, 2)
    try:
        sizes = [(1 << 17) - 1, 1 << 17, 700_001]
        ws = [inputs.by_name("exponential", n, 60 + n) for n in sizes]
        tks = [srv.build(torch.from_numpy(w).cuda()) for w in ws]
        bad = inputs.uniform(1 << 18, 9)
        bad[12345] = np.nan
        tbad = srv.build(torch.from_numpy(bad).cuda())
        for tk in tks:
            assert srv.wait(tk) == wrs.OK
        assert srv.wait(tbad) == wrs.ENONFINITE
        for w, tk in zip(ws, tks):
            assert torch.equal(served_rows(srv, tk, w.size), Built(w).rows_t.cpu())
        before = srv.stats()["resident_bytes"]
        assert srv.wait(srv.release(tks[2])) == wrs.OK
        assert srv.stats()["resident_bytes"] == before - 8 * sizes[2]
    finally:
        srv.close()
