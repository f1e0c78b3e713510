"""The precision study on the GPU: split and pack redone with FP64 or
paired-FP32 (compensated) prefix arithmetic (wrs_diag_prec_split_pack) on
the lists of an exact build.  The paper keeps these sums in FP64 (Sec. 2.2);
the oracle's study (oracle.psa_prec) shows both working types meet the
stated mass bound at these sizes, so each GPU variant's table must too:
|mass_i - N w_i/W| <= 1e-5 max(1, N w_i/W), with prob in [0, 1] and alias < N.
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle
import paper_2106_12270_gb300 as wrs
from paper_2106_12270_gb300 import inputs

pytestmark = pytest.mark.gpu

KINDS = ["uniform", "zipf", "exponential", "gamma"]
SIZES = [1, 2, 31, 1025, 4097, 100003]


def prec_table(w_np, prec, section=1024):
    n = w_np.size
    cfg = wrs.config(section)
    w = torch.from_numpy(w_np).cuda()
    ws = torch.empty(wrs.build_workspace_bytes(n, cfg), dtype=torch.uint8, device="cuda")
    pws = torch.empty(wrs.diag_prec_workspace_bytes(n, cfg), dtype=torch.uint8, device="cuda")
    rows = torch.zeros(n, dtype=torch.int64, device="cuda")
    info = torch.zeros(wrs.INFO_BYTES, dtype=torch.uint8, device="cuda")
    wrs.step_total(w, ws, cfg)
    wrs.step_partition(w, ws, cfg)
    wrs.diag_prec_split_pack(n, rows, ws, pws, cfg, prec)
    wrs.step_info(n, ws, info, cfg)
    torch.cuda.synchronize()
    return wrs.rows_to_numpy(rows), wrs.parse_info(info)


@pytest.mark.parametrize("prec", [wrs.PREC_FP64, wrs.PREC_FF])
@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("n", SIZES)
def test_prec_tables_meet_the_mass_bound(prec, kind, n):
    w = inputs.by_name(kind, n, 5000 + n)
    if w.sum() == 0:
        w[0] = 1.0
    (prob, alias), info = prec_table(w, prec)
    assert info["status"] == wrs.OK
    assert np.all((prob >= 0) & (prob <= 1)) and np.all(alias < n)
    W = oracle.exact_sum(w)
    assert oracle.mass_error(prob.astype(np.float64), alias, w, W) <= 1e-5


@pytest.mark.parametrize("section", [256, 512])
def test_prec_smaller_sections(section):
    w = inputs.by_name("zipf", 200003, 7)
    for prec in (wrs.PREC_FP64, wrs.PREC_FF):
        (prob, alias), info = prec_table(w, prec, section)
        assert info["status"] == wrs.OK
        W = oracle.exact_sum(w)
        assert oracle.mass_error(prob.astype(np.float64), alias, w, W) <= 1e-5


def test_prec_fp64_error_like_the_oracle_study():
    # 2e6 shuffled power law: the oracle's FP64 study table and the GPU's FP64
    # variant both sit at the FP32 rounding of the stored probabilities
    n = 2_000_000
    w = inputs.zipf_permuted(n, 3)
    W = oracle.exact_sum(w)
    p_orc, a_orc = oracle.psa_prec(w, 1024, oracle.PREC_FP64)
    e_orc = oracle.mass_error(p_orc.astype(np.float32).astype(np.float64), a_orc, w, W)
    (prob, alias), _ = prec_table(w, wrs.PREC_FP64)
    e_gpu = oracle.mass_error(prob.astype(np.float64), alias, w, W)
    assert e_gpu <= 1e-5 and e_orc <= 1e-5
    assert e_gpu <= 10 * max(e_orc, 1e-7)


def test_prec_rejects_large_sections():
    with pytest.raises(wrs.WrsError):
        wrs.diag_prec_workspace_bytes(1000, wrs.config(2048))
