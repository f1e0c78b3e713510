"""Parity of the CUDA sampling path with the CPU oracle (GPU required).

The GPU sampler and the oracle's sampler read the same exported GPU table
and the same Philox-4x32-10 counters, so the samples must agree bit for bit
(Sec. 2.2 Walker's rule in integer form).  The distribution itself is
checked by a chi-squared goodness-of-fit test at 1e8 draws.
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle
import paper_2106_12270_gb300 as wrs
from gpu_util import Built, gpu_sample
from paper_2106_12270_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def table_1e6():
    # plain single table: N = 1e6 uniform weights from seed 1
    return Built(inputs.uniform(1_000_000, 1))


@pytest.mark.parametrize("first, count, seed, slo, shi, offset", [
    (0, 10_000_000, 2, 0, 0, 0),
    (1, 1001, 2, 0, 0, 0),
    (12345, 777, 99, 7, 0, 1),
    (2**40 + 3, 5000, 2**63 + 5, 0xFFFFFFFF, 3, 3),
    (0, 1, 0, 0, 0, 1),
    (0, 0, 1, 0, 0, 0),
])
def test_naive_samples_bit_exact(table_1e6, first, count, seed, slo, shi, offset):
    b = table_1e6
    got = gpu_sample(b.rows_t, b.n, first, count, seed, slo, shi, offset)
    want = oracle.sample_naive(b.prob, b.alias, first, count, seed, slo, shi)
    assert np.array_equal(got, want)


def test_naive_chi_squared_1e8(table_1e6):
    from scipy import stats
    b = table_1e6
    n, draws = b.n, 100_000_000
    counts = torch.zeros(n, dtype=torch.int64, device="cuda")
    chunk = 10_000_000
    for first in range(0, draws, chunk):
        out = torch.empty(chunk, dtype=torch.int32, device="cuda")
        wrs.sample_rows(b.rows_t, n, first, chunk, 2, out)
        counts += torch.bincount(out.long(), minlength=n)
    c = counts.cpu().numpy()
    p = b.w.astype(np.float64) / b.w.astype(np.float64).sum()
    exp = p * draws
    # pool adjacent items until each pooled cell expects >= 5 draws
    order = np.arange(n)
    cells_o, cells_e, acc_o, acc_e = [], [], 0, 0.0
    for i in order:
        acc_o += c[i]
        acc_e += exp[i]
        if acc_e >= 5:
            cells_o.append(acc_o); cells_e.append(acc_e); acc_o, acc_e = 0, 0.0
    if acc_e > 0:
        cells_o[-1] += acc_o; cells_e[-1] += acc_e
    res = stats.chisquare(np.array(cells_o), np.array(cells_e) * (draws / sum(cells_e)))
    assert res.pvalue > 1e-3


@pytest.mark.parametrize("kind", ["zipf", "gamma"])
def test_naive_samples_other_tables(kind):
    b = Built(inputs.by_name(kind, 123457, 6))
    got = gpu_sample(b.rows_t, b.n, 5, 200_001, 11, 1, 0)
    want = oracle.sample_naive(b.prob, b.alias, 5, 200_001, 11, 1, 0)
    assert np.array_equal(got, want)


def test_naive_small_tables():
    for n in (1, 2, 3, 17):
        b = Built(inputs.exponential(n, n) + np.float32(0.01))
        got = gpu_sample(b.rows_t, n, 0, 10001, 3)
        want = oracle.sample_naive(b.prob, b.alias, 0, 10001, 3)
        assert np.array_equal(got, want)
        assert got.max() < n


def test_auto_choice_rule():
    assert wrs.sample_auto_choice(1000, 10**9) == "naive"          # tiny table in L2
    assert wrs.sample_auto_choice(1 << 27, 1000) == "naive"        # few draws
    assert wrs.sample_auto_choice(1 << 27, 1 << 28) == "cached"    # 2 draws per row
    assert wrs.sample_auto_choice(1 << 27, 1 << 24) == "cached"
    assert wrs.sample_auto_choice(1 << 24, 1 << 20) == "naive"
    assert wrs.sample_auto_choice(1 << 24, 1 << 28) == "smem"      # 16 draws per row
    assert wrs.sample_auto_choice(10**8, 10**9) == "smem"
    assert wrs.sample_auto_choice(1 << 20, 1 << 28) == "smem"      # 256 draws per row
    assert wrs.sample_auto_choice(1 << 20, 1 << 24) == "naive"


@pytest.mark.parametrize("n,count", [(100_003, 1_000_001), (1 << 23, 9_000_001),
                                     (1 << 23, 70_000_001)])
def test_auto_draws_exactly_what_the_chosen_mode_draws(n, count):
    w = inputs.by_name("zipf", n, 11)
    b = Built(w)
    out = torch.empty(count, dtype=torch.int32, device="cuda")
    mode = wrs.sample_auto(b.rows_t, n, count, 42, out)
    torch.cuda.synchronize()
    assert mode == wrs.sample_auto_choice(n, count)
    want = torch.empty_like(out)
    code, rows_per = wrs.sample_auto_plan(n, count)
    if mode == "naive":
        wrs.sample_rows(b.rows_t, n, 0, count, 42, want)
    else:
        nsec = wrs.sample_sections(n, rows_per)
        cnt = torch.empty(nsec, dtype=torch.int64, device="cuda")
        off = torch.empty(nsec, dtype=torch.int64, device="cuda")
        wrs.sample_sectioned_rows(b.rows_t, n, count, 42, code, rows_per, cnt, off, want)
    torch.cuda.synchronize()
    assert torch.equal(out, want)


@pytest.mark.parametrize("count, seed", [(1001, 0x0123456789ABCDEF), (4096, 2), (1, 7)])
def test_philox_probe_matches_oracle(count, seed):
    """The Philox-rate probe makes exactly the stated calls: out[2c] and
    out[2c+1] fold the four words of call c on counter (c, 0, 0, TAG_DIAG)."""
    out = torch.zeros(count + 1, dtype=torch.int32, device="cuda")
    wrs.diag_philox(count, seed, out)
    torch.cuda.synchronize()
    got = out.cpu().numpy().view(np.uint32)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    want = np.zeros(count + 1, np.uint32)
    for c in range((count + 1) // 2):
        x = oracle.philox([c & 0xFFFFFFFF, c >> 32, 0, wrs.TAG_DIAG], key)
        want[2 * c] = x[0] ^ x[1]
        if 2 * c + 1 < count:
            want[2 * c + 1] = x[2] ^ x[3]
    assert np.array_equal(got, want)   # including the untouched slot after count
