"""Sectioned sampling (Sec. 5) through the C ABI (GPU required).

The section counts come from the GPU (a random binomial split); given them,
the samples must equal the oracle's sectioned sampler bit for bit.  The
counts themselves are checked by their exact invariants (sum, offsets) and
statistically (multinomial chi-squared), and the whole stream by a
goodness-of-fit test against w/W.
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

MODES = [wrs.SAMPLE_CACHED, wrs.SAMPLE_LIMITED, wrs.SAMPLE_SMEM]


def run_sectioned(b, count, seed, mode, section_rows, offset=0):
    nsec = wrs.sample_sections(b.n, section_rows)
    counts = torch.zeros(nsec, dtype=torch.int64, device="cuda")
    offs = torch.zeros(nsec, dtype=torch.int64, device="cuda")
    buf = torch.empty(count + offset + 1, dtype=torch.int32, device="cuda")
    out = buf[offset: offset + count]
    wrs.sample_sectioned_rows(b.rows_t, b.n, count, seed, mode, section_rows, counts, offs, out)
    torch.cuda.synchronize()
    return (counts.cpu().numpy().astype(np.uint64), offs.cpu().numpy().astype(np.uint64),
            out.cpu().numpy().view(np.uint32))


@pytest.fixture(scope="module")
def table():
    return Built(inputs.zipf_permuted(1_000_003, 3))


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("section_rows, count, seed, offset", [
    (4096, 3_000_001, 5, 0),
    (16384, 1_000_000, 2**40 + 9, 1),
    (1000, 77, 1, 0),
    (1 << 21, 12345, 3, 0),    # one section: the whole table
])
def test_sectioned_bit_exact(table, mode, section_rows, count, seed, offset):
    if mode == wrs.SAMPLE_SMEM and section_rows > 24576:
        pytest.skip("SMEM mode holds a section in shared memory")
    counts, offs, out = run_sectioned(table, count, seed, mode, section_rows, offset)
    assert int(counts.sum()) == count
    assert np.array_equal(offs, np.concatenate([[0], np.cumsum(counts)[:-1]]).astype(np.uint64))
    want = oracle.sample_sectioned(table.prob, table.alias, counts, seed, wrs.TAG_SECTION)
    assert np.array_equal(out, want)


def test_modes_identical(table):
    res = [run_sectioned(table, 2_000_000, 17, m, 8192) for m in MODES]
    for r in res[1:]:
        assert np.array_equal(r[0], res[0][0]) and np.array_equal(r[2], res[0][2])


def test_counts_are_multinomial(table):
    from scipy import stats
    section_rows = 2048
    counts, _, _ = run_sectioned(table, 50_000_000, 23, wrs.SAMPLE_CACHED, section_rows)
    nsec = counts.size
    n = table.n
    rows = np.array([(s + 1) * n // nsec - s * n // nsec for s in range(nsec)], np.float64)
    exp = rows / n * counts.sum()
    assert stats.chisquare(counts.astype(np.float64), exp).pvalue > 1e-3


def test_small_counts_exact_path(table):
    # counts <= 96 per node use exact Bernoulli trials
    for count in (0, 1, 2, 95, 96, 97, 500):
        counts, offs, out = run_sectioned(table, count, 7, wrs.SAMPLE_CACHED, 4096)
        assert int(counts.sum()) == count
        want = oracle.sample_sectioned(table.prob, table.alias, counts, 7, wrs.TAG_SECTION)
        assert np.array_equal(out, want)


def test_sectioned_goodness_of_fit():
    from scipy import stats
    b = Built(inputs.uniform(200_000, 9))
    draws = 100_000_000
    counts, _, out = run_sectioned(b, draws, 31, wrs.SAMPLE_SMEM, 8192)
    c = np.bincount(out.astype(np.int64), minlength=b.n).astype(np.float64)
    p = b.w.astype(np.float64) / b.w.astype(np.float64).sum()
    exp = p * draws
    keep = exp >= 5
    res = stats.chisquare(c[keep], exp[keep] * (c[keep].sum() / exp[keep].sum()))
    assert res.pvalue > 1e-3


@pytest.mark.parametrize("n, section_rows", [(1, 1), (2, 1), (17, 4), (1000, 1)])
def test_sectioned_edge_tables(n, section_rows):
    b = Built(inputs.exponential(n, 4) + np.float32(0.01))
    counts, offs, out = run_sectioned(b, 10_001, 3, wrs.SAMPLE_SMEM, section_rows)
    assert int(counts.sum()) == 10_001
    want = oracle.sample_sectioned(b.prob, b.alias, counts, 3, wrs.TAG_SECTION)
    assert np.array_equal(out, want)


def test_sectioned_rejects_bad_arguments(table):
    nsec = wrs.sample_sections(table.n, 4096)
    counts = torch.zeros(nsec, dtype=torch.int64, device="cuda")
    out = torch.empty(10, dtype=torch.int32, device="cuda")
    with pytest.raises(wrs.WrsError):
        wrs.sample_sectioned_rows(table.rows_t, table.n, 10, 1, wrs.SAMPLE_SMEM, 100_000,
                                  counts, counts, out)
    with pytest.raises(wrs.WrsError):
        wrs.sample_sectioned_rows(table.rows_t, table.n, 10, 1, 9, 4096, counts, counts, out)
