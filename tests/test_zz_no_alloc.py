"""The allocation-free build entry point (wrs_build_rows_noalloc), GPU.

It serves callers that cannot allocate device memory at build time (a fixed
start-up memory plan, or a framework that owns the allocator); its
workspace is a fixed array inside the library.  Two calls in a row, on
different inputs, must give exactly the tables the regular entry point
(wrs_build_rows with a caller workspace) gives -- so nothing the first call
leaves in the shared array leaks into the second -- and sizes beyond the
array's limit must be refused.  This file is collected last on purpose.
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle
import paper_2106_12270_gb300 as wrs
from paper_2106_12270_gb300 import inputs

pytestmark = pytest.mark.gpu


def regular(w):
    b = wrs.Builder(w.numel())
    rows = b.build(w)
    torch.cuda.synchronize()
    return rows, wrs.parse_info(b.info)


def noalloc(w):
    rows = torch.empty(w.numel(), dtype=torch.int64, device="cuda")
    info = torch.zeros(wrs.INFO_BYTES, dtype=torch.uint8, device="cuda")
    wrs.build_rows_noalloc(w, rows, info)
    torch.cuda.synchronize()
    return rows, wrs.parse_info(info)


def test_noalloc_matches_regular_on_two_calls_in_a_row():
    cases = [inputs.uniform(1_000_003, 1), inputs.zipf_permuted(777_777, 3)]
    for w_np in cases:
        w = torch.from_numpy(w_np).cuda()
        want_rows, want_info = regular(w)
        got_rows, got_info = noalloc(w)
        assert got_info == want_info
        assert got_info["status"] == wrs.OK
        assert torch.equal(got_rows, want_rows)
        prob, alias = wrs.rows_to_numpy(got_rows)
        W = oracle.exact_sum(w_np)
        assert oracle.mass_error(prob.astype(np.float64), alias, w_np, W) <= 1e-5


def test_noalloc_refuses_sizes_beyond_its_array():
    w = torch.ones(3_500_001, device="cuda")
    rows = torch.empty(w.numel(), dtype=torch.int64, device="cuda")
    info = torch.zeros(wrs.INFO_BYTES, dtype=torch.uint8, device="cuda")
    with pytest.raises(wrs.WrsError) as e:
        wrs.build_rows_noalloc(w, rows, info)
    assert e.value.status == wrs.EINVAL
