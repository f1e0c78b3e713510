"""Batched construction and sampling of many tables in one launch (GPU).

Every table of a batch must be the very table the single-table path builds
for the same weights (same exact arithmetic: bit-identical rows), match the
oracle (exact W, light/heavy counts, mass within 1e-5), and its samples must
equal the oracle's sampler on stream (table, WRS_TAG_BATCH) bit for bit.
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle
import paper_2106_12270_gb300 as wrs
from gpu_util import Built
from paper_2106_12270_gb300 import inputs

pytestmark = pytest.mark.gpu


def build_batch(w_np, off_np, order=True):
    ntab = off_np.size - 1
    w = torch.from_numpy(np.ascontiguousarray(w_np, np.float32)).cuda()
    off = torch.from_numpy(off_np.astype(np.int64)).cuda()
    rows = torch.zeros(max(int(off_np[-1]), 1), dtype=torch.int64, device="cuda")
    bb = wrs.BatchBuilder(int(off_np[-1]), ntab)
    ord_t = torch.from_numpy(wrs.batch_order(off_np).astype(np.int32)).cuda() if order else None
    bb.build(w, off, rows, ord_t)
    torch.cuda.synchronize()
    return rows, bb.summaries(), off


@pytest.fixture(scope="module")
def batch():
    sizes = inputs.log_uniform_sizes(300, 6, 16, 65536)
    sizes[:4] = [1, 2, 4096, 4097]   # tiny tables and a partition-tile boundary
    w, off = inputs.batched(sizes, 7, "gamma")
    rows, summ, off_t = build_batch(w, off)
    return w, off, rows, summ, off_t


def table_rows(rows, off, t):
    prob, alias = wrs.rows_to_numpy(rows[int(off[t]): int(off[t + 1])])
    return prob, alias


def test_batched_matches_oracle(batch):
    w, off, rows, summ, _ = batch
    for t in range(off.size - 1):
        wt = w[off[t]: off[t + 1]]
        if wt.sum() == 0:
            assert summ[t]["status"] == wrs.EZEROSUM
            continue
        W = oracle.exact_sum(wt)
        assert summ[t]["status"] == wrs.OK
        assert summ[t]["W"] == W
        l, h = oracle.classify(wt, W / wt.size)
        assert (summ[t]["nl"], summ[t]["nh"]) == (len(l), len(h))
        prob, alias = table_rows(rows, off, t)
        assert np.all(alias < wt.size)
        assert oracle.mass_error(prob.astype(np.float64), alias, wt, W) <= 1e-5


def test_batched_equals_single_table_builds(batch):
    w, off, rows, summ, _ = batch
    for t in list(range(0, off.size - 1, 7)) + [2, 3]:
        wt = w[off[t]: off[t + 1]]
        if wt.sum() == 0:
            continue
        b = Built(wt)
        prob, alias = table_rows(rows, off, t)
        assert np.array_equal(prob.view(np.uint32), b.prob.view(np.uint32)), t
        assert np.array_equal(alias, b.alias), t


def test_batched_order_does_not_matter(batch):
    w, off, rows, summ, _ = batch
    rows2, summ2, _ = build_batch(w, off, order=False)
    assert torch.equal(rows, rows2)
    assert np.array_equal(summ["W"], summ2["W"])


def test_batched_sampling_bit_exact(batch):
    w, off, rows, summ, off_t = batch
    ntab = off.size - 1
    cnt = np.full(ntab, 1001, np.int64)
    cnt[5] = 0
    cnt_off = np.zeros(ntab + 1, np.int64)
    cnt_off[1:] = np.cumsum(cnt)
    out = torch.empty(int(cnt_off[-1]), dtype=torch.int32, device="cuda")
    wrs.sample_batched_rows(rows, off_t, ntab, torch.from_numpy(cnt_off).cuda(), 99, out)
    torch.cuda.synchronize()
    got = out.cpu().numpy().view(np.uint32)
    for t in range(0, ntab, 11):
        if summ[t]["status"] != wrs.OK:
            continue
        prob, alias = table_rows(rows, off, t)
        want = oracle.sample_naive(prob, alias, 0, int(cnt[t]), 99, t, wrs.TAG_BATCH)
        assert np.array_equal(got[cnt_off[t]: cnt_off[t + 1]], want), t


def test_batched_bad_tables_do_not_spoil_others():
    sizes = np.array([100, 0, 50, 30, 70])
    w, off = inputs.batched(sizes, 3, "uniform")
    w[off[2] + 5] = np.nan
    w[off[3]: off[4]] = 0.0
    w[off[4] + 1] = -1.0
    rows, summ, _ = build_batch(w, off)
    assert summ["status"].tolist() == [wrs.OK, wrs.EINVAL, wrs.ENONFINITE, wrs.EZEROSUM,
                                       wrs.EINVAL]
    prob, alias = table_rows(rows, off, 0)
    W = oracle.exact_sum(w[:100])
    assert oracle.mass_error(prob.astype(np.float64), alias, w[:100], W) <= 1e-5


TILINGS = [(t, c) for t in (256, 512) for c in (512, 1024, 2048, 4096)]


@pytest.mark.parametrize("threads,chunk", TILINGS)
def test_every_tiling_builds_the_same_tables(batch, threads, chunk):
    """The tiling only changes the time: rows and summaries of the chunked
    kernel are bit-identical to the default (segmented) build's."""
    w, off, rows, summ, off_t = batch
    wt = torch.from_numpy(np.ascontiguousarray(w, np.float32)).cuda()
    rows2 = torch.zeros_like(rows)
    bb = wrs.BatchBuilder(int(off[-1]), off.size - 1)
    bb.tuning = wrs.BatchTuning(threads, chunk, 0, 0.0)
    bb.build(wt, off_t, rows2, None)
    torch.cuda.synchronize()
    assert torch.equal(rows, rows2)
    assert np.array_equal(summ.view(np.uint8), bb.summaries().view(np.uint8))


def test_invalid_tiling_rejected(batch):
    w, off, rows, summ, off_t = batch
    wt = torch.from_numpy(np.ascontiguousarray(w, np.float32)).cuda()
    bb = wrs.BatchBuilder(int(off[-1]), off.size - 1)
    for bad in ((128, 1024), (256, 8192), (300, 1024), (0, 1024)):
        bb.tuning = wrs.BatchTuning(bad[0], bad[1], 0, 0.0)
        with pytest.raises(wrs.WrsError):
            bb.build(wt, off_t, torch.zeros_like(rows), None)


def test_autotune_picks_a_candidate_and_caches_it(batch):
    w, off, rows, summ, off_t = batch
    wt = torch.from_numpy(np.ascontiguousarray(w, np.float32)).cuda()
    rows2 = torch.zeros_like(rows)
    bb = wrs.BatchBuilder(int(off[-1]), off.size - 1)
    best, cand = bb.autotune(wt, off_t, rows2, None, force=True)
    # the segmented build (threads 0) and every tiling of the chunked kernel
    assert len(cand) == len(TILINGS) + 1
    assert {(c["threads"], c["chunk"]) for c in cand} == set(TILINGS) | {(0, 0)}
    assert all(c["ms"] > 0 for c in cand)
    assert best["ms"] == min(c["ms"] for c in cand)
    assert torch.equal(rows, rows2)            # the buffers hold a valid build
    again, cand2 = bb.autotune(wt, off_t, rows2, None)   # cached: no timing
    assert cand2 == [] and (again["threads"], again["chunk"]) == (best["threads"], best["chunk"])


def test_batched_build_and_sample_replay_as_cuda_graph(batch):
    """One captured graph (build + sample) replays to the eager results."""
    w, off, rows, summ, off_t = batch
    ntab = off.size - 1
    wt = torch.from_numpy(np.ascontiguousarray(w, np.float32)).cuda()
    cnt_off = torch.arange(0, 501 * (ntab + 1), 501, dtype=torch.int64, device="cuda")
    bb = wrs.BatchBuilder(int(off[-1]), ntab)
    rows_g = torch.zeros_like(rows)
    out_g = torch.empty(int(cnt_off[-1]), dtype=torch.int32, device="cuda")
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):   # warm-up outside the capture (kernel attributes)
        bb.build(wt, off_t, rows_g, None, stream=s)
        wrs.sample_batched_rows(rows_g, off_t, ntab, cnt_off, 5, out_g, stream=s)
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        st = torch.cuda.current_stream()
        bb.build(wt, off_t, rows_g, None, stream=st)
        wrs.sample_batched_rows(rows_g, off_t, ntab, cnt_off, 5, out_g, stream=st)
    rows_g.zero_()
    out_g.zero_()
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(rows_g, rows)
    out_e = torch.empty_like(out_g)
    wrs.sample_batched_rows(rows, off_t, ntab, cnt_off, 5, out_e)
    torch.cuda.synchronize()
    assert torch.equal(out_g, out_e)


def _edge_tables():
    """Tables around chunk sizes and with extreme light/heavy mixes: the
    chunked sweep's windows run out of lights first, of heavies first, or
    end exactly on a chunk."""
    r = np.random.default_rng(31)
    tabs = []
    for n in (511, 512, 513, 1023, 1024, 1025, 2047, 2048, 2049, 4095, 4096, 4097, 8193):
        tabs.append(r.random(n).astype(np.float32))                       # uniform
        tabs.append(r.exponential(1.0, n).astype(np.float32))              # Exp(1)
    for n in (3000, 9000):
        w = np.ones(n, np.float32)
        w[r.random(n) < 0.1] = 0.01        # 90% heavy: lights run out first
        tabs.append(w)
        w = np.ones(n, np.float32)
        w[n // 3] = 1e6                    # one heavy that fills everything
        tabs.append(w)
        tabs.append(np.full(n, 0.37, np.float32))                          # all light
        tabs.append((1.0 + r.integers(-64, 64, n) * 2.0**-23).astype(np.float32))
        w = r.gamma(0.1, 1.0, n).astype(np.float32)
        w[: n // 2] = 0.0                  # a long run of zero weights
        tabs.append(w)
    return tabs


@pytest.mark.parametrize("threads,chunk", [(256, 1024), (256, 512), (512, 2048)])
def test_batched_window_edges_equal_single_builds(threads, chunk):
    tabs = _edge_tables()
    sizes = np.array([t.size for t in tabs], np.int64)
    off = np.zeros(sizes.size + 1, np.uint64)
    off[1:] = np.cumsum(sizes).astype(np.uint64)
    w = np.concatenate(tabs)
    wt = torch.from_numpy(w).cuda()
    off_t = torch.from_numpy(off.astype(np.int64)).cuda()
    rows = torch.zeros(int(off[-1]), dtype=torch.int64, device="cuda")
    bb = wrs.BatchBuilder(int(off[-1]), sizes.size)
    bb.tuning = wrs.BatchTuning(threads, chunk, 0, 0.0)
    bb.build(wt, off_t, rows, None)
    torch.cuda.synchronize()
    summ = bb.summaries()
    for t, wtab in enumerate(tabs):
        assert summ[t]["status"] == wrs.OK, t
        b = Built(wtab)
        prob, alias = table_rows(rows, off, t)
        assert np.array_equal(prob.view(np.uint32), b.prob.view(np.uint32)), t
        assert np.array_equal(alias, b.alias), t


@pytest.mark.parametrize("sizes", [[1 << 20 | 7, 1024, 1025, 2048, 3, 300001, 65536],
                                   [5000] * 40 + [1 << 18]])
def test_segmented_build_equals_single_builds(sizes):
    """The segmented build (each table's lists and checkpoints by one CTA,
    then the single-table split and pack over every table's sections of 1024
    buckets): every table bit-identical to the single-table build of its
    weights, with tables of one and of many sections, ragged and exact."""
    sizes = np.asarray(sizes, np.int64)
    w, off = inputs.batched(sizes, 23, "exponential")
    rows, summ, _ = build_batch(w, off)
    for t in range(sizes.size):
        wt = w[off[t]: off[t + 1]]
        b = Built(wt)
        assert summ[t]["status"] == wrs.OK
        assert (summ[t]["W"], summ[t]["nl"], summ[t]["nh"]) == \
            (b.info["W"], b.info["nl"], b.info["nh"])
        prob, alias = table_rows(rows, off, t)
        assert np.array_equal(prob.view(np.uint32), b.prob.view(np.uint32)), t
        assert np.array_equal(alias, b.alias), t


def test_bad_tables_on_both_partition_paths():
    """Bad tables among large ones (a CTA each, more than 8192 items) and
    small ones (a warp each, statistics then placement): each reports its
    status, and every good table is the single-table build bit for bit."""
    sizes = np.array([20000, 100, 20011, 50, 30000, 7, 40000, 64], np.int64)
    w, off = inputs.batched(sizes, 29, "gamma")
    w[off[0] + 17] = np.nan          # large: non-finite
    w[off[3] + 3] = -2.0             # small: negative
    w[off[4]: off[5]] = 0.0          # large: zero total
    w[off[5] + 2] = np.inf           # small: non-finite
    w[off[6] + 39999] = -0.5         # large: negative, its last item
    rows, summ, _ = build_batch(w, off)
    want = [wrs.ENONFINITE, wrs.OK, wrs.OK, wrs.EINVAL, wrs.EZEROSUM, wrs.ENONFINITE,
            wrs.EINVAL, wrs.OK]
    assert summ["status"].tolist() == want
    for t in np.flatnonzero(np.array(want) == wrs.OK):
        wt = w[off[t]: off[t + 1]]
        b = Built(wt)
        assert (summ[t]["W"], summ[t]["nl"], summ[t]["nh"]) == \
            (b.info["W"], b.info["nl"], b.info["nh"])
        prob, alias = table_rows(rows, off, t)
        assert np.array_equal(prob.view(np.uint32), b.prob.view(np.uint32)), t
        assert np.array_equal(alias, b.alias), t


def test_segmented_build_workspace_too_small():
    """A workspace laid out for fewer items than the batch holds: the tables
    that do not fit report WRS_EINVAL, the others are built."""
    sizes = np.asarray([40000, 30000, 20000, 10000], np.int64)
    w, off = inputs.batched(sizes, 29, "uniform")
    wt = torch.from_numpy(w).cuda()
    off_t = torch.from_numpy(off.astype(np.int64)).cuda()
    rows = torch.zeros(int(off[-1]), dtype=torch.int64, device="cuda")
    bb = wrs.BatchBuilder(70000, sizes.size)   # room for the first two tables
    bb.build(wt, off_t, rows, None)
    torch.cuda.synchronize()
    summ = bb.summaries()
    assert summ["status"].tolist()[:2] == [wrs.OK, wrs.OK]
    assert summ["status"].tolist()[2:] == [wrs.EINVAL, wrs.EINVAL]
    for t in range(2):
        b = Built(w[off[t]: off[t + 1]])
        prob, alias = table_rows(rows, off, t)
        assert np.array_equal(prob.view(np.uint32), b.prob.view(np.uint32))
        assert np.array_equal(alias, b.alias)
