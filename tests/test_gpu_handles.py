"""The table and batch objects of the C ABI (wrs_build, wrs_sample,
wrs_table_*, wrs_build_batched, wrs_sample_batched, wrs_batch_*), GPU.

They are the problem statement's interface (Sec. 1: build(weights) ->
table, sample(table, count, seed) -> indices) over the buffer calls, so
their results must equal the buffer calls' bit for bit, and through them the
oracle's: the naive samples equal the oracle's sampler on the exported table.
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle
import paper_2106_12270_gb300 as wrs
from paper_2106_12270_gb300 import inputs

pytestmark = pytest.mark.gpu


def buffer_build(w, cfg=None):
    b = wrs.Builder(w.numel(), cfg)
    rows = b.build(w)
    torch.cuda.synchronize()
    return rows, wrs.parse_info(b.info)


@pytest.mark.parametrize("source", ["device", "host", "pinned"])
@pytest.mark.parametrize("kind,n", [("uniform", 1), ("zipf", 5000), ("gamma", 100_003)])
def test_table_build_equals_buffer_build(source, kind, n):
    w_np = inputs.by_name(kind, n, 40 + n)
    if w_np.sum() == 0:
        w_np[0] = 1.0
    w_dev = torch.from_numpy(w_np).cuda()
    want_rows, want_info = buffer_build(w_dev)
    arg = {"device": w_dev, "host": torch.from_numpy(w_np),
           "pinned": torch.from_numpy(w_np).pin_memory()}[source]
    t = wrs.Table.build(arg)
    info = t.info()
    assert (info["n"], info["W"], info["nl"], info["nh"]) == \
        (n, want_info["W"], want_info["nl"], want_info["nh"])
    assert info["W"] == oracle.exact_sum(w_np)
    assert torch.equal(t.export(device=True), want_rows)
    assert torch.equal(t.export(), want_rows.cpu())
    t.close()


def test_table_sampling_modes_equal_buffer_calls():
    n = 300_007
    w_np = inputs.exponential(n, 4)
    t = wrs.Table.build(w_np)
    rows = t.export(device=True)
    count = 2_000_001
    got = torch.empty(count, dtype=torch.int32, device="cuda")
    want = torch.empty(count, dtype=torch.int32, device="cuda")
    # naive: stream (seed, 0, TAG_NAIVE), as the oracle's sampler
    t.sample(count, 9, got, wrs.SAMPLE_NAIVE)
    wrs.sample_rows(rows, n, 0, count, 9, want)
    torch.cuda.synchronize()
    assert torch.equal(got, want)
    prob, alias = wrs.rows_to_numpy(rows)
    assert np.array_equal(got[:100_000].cpu().numpy().view(np.uint32),
                          oracle.sample_naive(prob, alias, 0, 100_000, 9))
    # sectioned modes: 8192 rows per section (cached, limited), 4096 (smem)
    for mode, sec_rows in ((wrs.SAMPLE_CACHED, 8192), (wrs.SAMPLE_LIMITED, 8192),
                           (wrs.SAMPLE_SMEM, 4096)):
        nsec = wrs.sample_sections(n, sec_rows)
        cnt = torch.empty(nsec, dtype=torch.int64, device="cuda")
        off = torch.empty(nsec, dtype=torch.int64, device="cuda")
        t.sample(count, 9, got, mode)
        wrs.sample_sectioned_rows(rows, n, count, 9, mode, sec_rows, cnt, off, want)
        torch.cuda.synchronize()
        assert torch.equal(got, want), mode
    # AUTO: the mode wrs_sample_auto picks, same output
    t.sample(count, 9, got, wrs.SAMPLE_AUTO)
    wrs.sample_auto(rows, n, count, 9, want)
    torch.cuda.synchronize()
    assert torch.equal(got, want)
    t.close()


def test_export_import_round_trip():
    n = 65_537
    w_np = inputs.gamma(n, 3)
    t = wrs.Table.build(w_np)
    host_rows = t.export()
    t2 = wrs.Table.import_rows(host_rows, t.info()["W"])
    t3 = wrs.Table.import_rows(host_rows.cuda(), t.info()["W"])
    a = torch.empty(1_000_000, dtype=torch.int32, device="cuda")
    b = torch.empty_like(a)
    c = torch.empty_like(a)
    t.sample(a.numel(), 5, a)
    t2.sample(b.numel(), 5, b)
    t3.sample(c.numel(), 5, c)
    torch.cuda.synchronize()
    assert torch.equal(a, b) and torch.equal(a, c)
    assert t2.info()["W"] == t.info()["W"]
    for x in (t, t2, t3):
        x.close()


def test_import_rejects_invalid_rows():
    good = wrs.Table.build(inputs.uniform(1000, 1)).export()
    raw = good.numpy().view(np.uint32).reshape(-1, 2)
    bad_prob = raw.copy()
    bad_prob[17, 0] = np.float32(1.5).view(np.uint32)
    bad_alias = raw.copy()
    bad_alias[3, 1] = 1000
    for arr in (bad_prob, bad_alias):
        rows = torch.from_numpy(arr.reshape(-1).view(np.int64).copy())
        with pytest.raises(wrs.WrsError) as e:
            wrs.Table.import_rows(rows)
        assert e.value.status == wrs.EINVAL


@pytest.mark.parametrize("bad,status", [(-1.0, wrs.EINVAL), (float("nan"), wrs.ENONFINITE),
                                        (float("inf"), wrs.ENONFINITE)])
def test_table_build_reports_data_errors(bad, status):
    w = inputs.uniform(5000, 2)
    w[1234] = bad
    with pytest.raises(wrs.WrsError) as e:
        wrs.Table.build(w)
    assert e.value.status == status
    with pytest.raises(wrs.WrsError) as e:
        wrs.Table.build(np.zeros(100, np.float32))
    assert e.value.status == wrs.EZEROSUM


def test_set_config_applies_to_table_builds():
    w_np = inputs.zipf_permuted(50_000, 3)
    w = torch.from_numpy(w_np).cuda()
    old = wrs.get_config()
    try:
        cfg = wrs.config(2048, wrs.SPLIT_BINARY)
        wrs.set_config(cfg)
        got = wrs.get_config()
        assert (got.section_size, got.split_method) == (2048, wrs.SPLIT_BINARY)
        want_rows, _ = buffer_build(w, cfg)
        t = wrs.Table.build(w)
        assert torch.equal(t.export(device=True), want_rows)
        t.close()
    finally:
        wrs.set_config(old)


def test_batch_objects_equal_batched_buffer_calls():
    sizes = inputs.log_uniform_sizes(500, 6, 16, 65536)
    sizes[:3] = [1, 2, 4097]
    w_np, off_np = inputs.batched(sizes, 7, "gamma")
    zero = 5
    w_np[off_np[zero]:off_np[zero + 1]] = 0.0   # one all-zero table: EZEROSUM
    total = int(off_np[-1])
    w = torch.from_numpy(w_np).cuda()
    off = torch.from_numpy(off_np.astype(np.int64)).cuda()
    ntab = sizes.size
    want = torch.zeros(total, dtype=torch.int64, device="cuda")
    bb = wrs.BatchBuilder(total, ntab)
    bb.build(w, off, want)
    torch.cuda.synchronize()
    summ_want = bb.summaries()
    b = wrs.Batch.build(w, off)
    assert b.ntab == ntab
    got = b.export(torch.zeros(total, dtype=torch.int64, device="cuda"))
    ok = summ_want["status"] == wrs.OK
    assert np.array_equal(b.status(), summ_want["status"])
    assert b.status()[zero] == wrs.EZEROSUM
    summ = b.summaries()
    assert np.array_equal(summ["W"][ok], summ_want["W"][ok])
    # rows of the tables that were built (the failed one is left untouched)
    for t in np.flatnonzero(ok):
        a, z = int(off_np[t]), int(off_np[t + 1])
        assert torch.equal(got[a:z], want[a:z]), t
    # the per-table baseline (one launch sequence per table) builds the same rows
    each = torch.zeros(total, dtype=torch.int64, device="cuda")
    _, nbad = wrs.diag_build_each(w, off_np, each, 1)
    assert nbad == 1
    for t in np.flatnonzero(ok):
        a, z = int(off_np[t]), int(off_np[t + 1])
        assert torch.equal(each[a:z], want[a:z]), t
    # batched sampling through the object equals the buffer call
    cnt_off = torch.arange(0, (ntab + 1) * 100, 100, dtype=torch.int64, device="cuda")
    s1 = torch.empty(ntab * 100, dtype=torch.int32, device="cuda")
    s2 = torch.empty_like(s1)
    b.sample(cnt_off, 11, s1)
    wrs.sample_batched_rows(want, off, ntab, cnt_off, 11, s2)
    torch.cuda.synchronize()
    for t in np.flatnonzero(ok):
        assert torch.equal(s1[100 * t:100 * (t + 1)], s2[100 * t:100 * (t + 1)]), t
    b.close()
