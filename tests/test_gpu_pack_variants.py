"""The paper's sequential pack designs (Sec. 4.2, Fig. 3) against the
production merge-path pack (GPU required).

Every variant sweeps each section from the same split state with the same
comparison rule, so its rows must equal step_pack's bit for bit; the pack's
own rows are checked against the oracle in test_gpu_build.py.
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle
import paper_2106_12270_gb300 as wrs
from paper_2106_12270_gb300 import inputs

pytestmark = pytest.mark.gpu

VARIANTS = [0, 1, 2]


def packed(w_np, section, variants):
    w_np = np.ascontiguousarray(w_np, np.float32)
    n = w_np.size
    cfg = wrs.config(section)
    w = torch.from_numpy(w_np).cuda()
    ws = torch.empty(wrs.build_workspace_bytes(n, cfg), dtype=torch.uint8, device="cuda")
    wrs.step_total(w, ws, cfg)
    wrs.step_partition(w, ws, cfg)
    wrs.step_split(n, ws, cfg)
    ref = torch.empty(n, dtype=torch.int64, device="cuda")
    wrs.step_pack(n, ref, ws, cfg)
    info = torch.zeros(wrs.INFO_BYTES, dtype=torch.uint8, device="cuda")
    wrs.step_info(n, ws, info, cfg)
    out = {}
    for v in variants:
        rows = torch.full((n,), -1, dtype=torch.int64, device="cuda")
        wrs.diag_pack_variant(w if v == 0 else None, n, rows, ws, cfg, v)
        out[v] = rows
    torch.cuda.synchronize()
    return ref.cpu(), {v: r.cpu() for v, r in out.items()}, wrs.parse_info(info)


@pytest.mark.parametrize("kind", ["uniform", "zipf", "exponential", "gamma"])
@pytest.mark.parametrize("n", [1, 2, 33, 1023, 4097, 100003])
def test_variants_equal_pack(kind, n):
    w = inputs.by_name(kind, n, 500 + n)
    if w.sum() == 0:
        w[0] = 1.0
    ref, out, info = packed(w, 1024, VARIANTS)
    assert info["status"] == wrs.OK
    for v in VARIANTS:
        assert torch.equal(out[v], ref), v


@pytest.mark.parametrize("section", [256, 2048, 8192])
def test_variants_every_section_size(section):
    n = 300007
    w = inputs.by_name("exponential", n, 77)
    ref, out, info = packed(w, section, VARIANTS)
    assert info["status"] == wrs.OK
    for v in VARIANTS:
        assert torch.equal(out[v], ref), v
    # and the table is a valid one for w
    raw = ref.numpy().view(np.uint32).reshape(-1, 2)
    m = oracle.mass(raw[:, 0].view(np.float32).astype(np.float64), raw[:, 1])
    e = oracle.expected_mass(w, oracle.exact_sum(w))
    assert float((np.abs(m - e) / np.maximum(1.0, e)).max()) <= 1e-5


def test_variants_degenerate():
    # all lights (equal weights) and one dominant heavy
    for w in (np.full(5000, 0.25, np.float32),
              np.concatenate([np.ones(4999, np.float32), np.float32([1e6])])):
        ref, out, info = packed(w, 1024, VARIANTS)
        assert info["status"] == wrs.OK
        for v in VARIANTS:
            assert torch.equal(out[v], ref), v


def test_variant_rejects_bad_arguments():
    n = 1000
    cfg = wrs.config()
    ws = torch.empty(wrs.build_workspace_bytes(n, cfg), dtype=torch.uint8, device="cuda")
    rows = torch.empty(n, dtype=torch.int64, device="cuda")
    with pytest.raises(wrs.WrsError) as e:
        wrs.diag_pack_variant(None, n, rows, ws, cfg, 3)
    assert e.value.status == wrs.EINVAL
    with pytest.raises(wrs.WrsError) as e:
        wrs.diag_pack_variant(None, n, rows, ws, cfg, 0)   # the gather needs the weights
    assert e.value.status == wrs.EINVAL
