"""The allocation-free build entry point (wrs_build_rows_noalloc), GPU.

It serves callers that cannot allocate device memory at build time (a fixed
start-up memory plan, or a framework that owns the allocator); its
workspace is a fixed array inside the library, shared by every call on a
device.  Calls in a row, on different inputs and sizes (larger, smaller,
larger again, and the largest size it accepts), must give exactly the tables
the regular entry point (wrs_build_rows with a caller workspace) gives -- so
nothing an earlier call leaves in the shared array leaks into a later one --
and sizes beyond the array's limit must be refused.

The file name sorts last so that a run stopping at its first failure has
already run every other test before this one; it also passes alone in a
fresh process (the array needs no set-up by an earlier test).
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle
import paper_2106_12270_gb300 as wrs
from paper_2106_12270_gb300 import inputs

pytestmark = pytest.mark.gpu

MAX_ITEMS = 3_500_000


def regular(w, cfg=None):
    b = wrs.Builder(w.numel(), cfg)
    rows = b.build(w)
    torch.cuda.synchronize()
    return rows, wrs.parse_info(b.info)


def noalloc(w, cfg=None):
    rows = torch.empty(w.numel(), dtype=torch.int64, device="cuda")
    info = torch.zeros(wrs.INFO_BYTES, dtype=torch.uint8, device="cuda")
    wrs.build_rows_noalloc(w, rows, info, cfg)
    torch.cuda.synchronize()
    return rows, wrs.parse_info(info)


def check_same(w_np, cfg=None):
    w = torch.from_numpy(w_np).cuda()
    want_rows, want_info = regular(w, cfg)
    got_rows, got_info = noalloc(w, cfg)
    assert got_info == want_info
    assert got_info["status"] == wrs.OK
    assert torch.equal(got_rows, want_rows)
    prob, alias = wrs.rows_to_numpy(got_rows)
    W = oracle.exact_sum(w_np)
    assert oracle.mass_error(prob.astype(np.float64), alias, w_np, W) <= 1e-5


def test_noalloc_matches_regular_on_calls_in_a_row():
    # larger, smaller, then larger again with skewed weights (the earlier
    # calls' leftovers lie inside the live regions of the last one), then the
    # same size twice
    for w_np in (inputs.uniform(1_000_003, 1), inputs.zipf_permuted(777_777, 3),
                 inputs.gamma(2_500_001, 7), inputs.gamma(2_500_001, 8)):
        check_same(w_np)


def test_noalloc_largest_size_with_smallest_sections():
    # the largest accepted n with the section size whose workspace is largest
    check_same(inputs.exponential(MAX_ITEMS, 4), wrs.config(256))


def test_noalloc_refuses_sizes_beyond_its_array():
    w = torch.ones(MAX_ITEMS + 1, device="cuda")
    rows = torch.empty(w.numel(), dtype=torch.int64, device="cuda")
    info = torch.zeros(wrs.INFO_BYTES, dtype=torch.uint8, device="cuda")
    with pytest.raises(wrs.WrsError) as e:
        wrs.build_rows_noalloc(w, rows, info)
    assert e.value.status == wrs.EINVAL
