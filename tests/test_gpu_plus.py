"""PSA+ construction (Sec. 4 "PSA+") on the GPU against the CPU oracle.

The greedy step packs each tile of 1024 consecutive items that holds at
least `min_items` lights and heavies; the rest goes through PSA.  The GPU table is
not the oracle's row for row (the rest's PSA recomputes its own total in FP32
weights, the oracle keeps the FP64 average), so parity is checked on:
* the reconstructed masses: |mass_i - N w_i/W| <= 1e-5 max(1, N w_i/W);
* the number of items the greedy step finished: equal to the oracle's
  psa_plus with tiles of 1024 (the two sweeps decide at different
  resolutions -- the oracle in FP64, the GPU on exact prefixes at 2^-46 of a
  bucket -- so only an exact near-tie could separate them, and none occurs on
  these seeded inputs);
* rows bit-identical to the PSA build when no chunk is eligible;
* status codes of the whole-table steps.
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle
import paper_2106_12270_gb300 as wrs
from paper_2106_12270_gb300 import inputs

pytestmark = pytest.mark.gpu

MASS_TOL = 1e-5
TILE = 1024
KINDS = ["uniform", "zipf", "exponential", "gamma"]
SIZES = [1, 2, 3, 1023, 1024, 1025, 4097, 100003]


def build_plus(w_np, min_items=1, cfg=None, offset=0):
    """One PSA+ build through the C ABI; returns (prob, alias, info, greedy)."""
    w = np.ascontiguousarray(w_np, np.float32)
    n = w.size
    cfg = cfg if cfg is not None else wrs.config()
    buf = torch.zeros(n + offset, dtype=torch.float32, device="cuda")
    buf[offset:] = torch.from_numpy(w).cuda()
    w_dev = buf[offset:]
    rows = torch.empty(n, dtype=torch.int64, device="cuda")
    ws = torch.empty(wrs.build_plus_workspace_bytes(n, cfg), dtype=torch.uint8, device="cuda")
    info = torch.zeros(wrs.INFO_BYTES, dtype=torch.uint8, device="cuda")
    greedy = wrs.build_rows_plus(w_dev, rows, ws, info, cfg, min_items)
    torch.cuda.synchronize()
    inf = wrs.parse_info(info)
    prob, alias = wrs.rows_to_numpy(rows) if inf["status"] == wrs.OK else (None, None)
    return prob, alias, inf, greedy


def mass_err(w, prob, alias):
    e = oracle.expected_mass(w, oracle.exact_sum(w))
    m = oracle.mass(prob.astype(np.float64), alias)
    return float((np.abs(m - e) / np.maximum(1.0, e)).max())


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("n", SIZES)
def test_plus_masses_and_greedy_count(kind, n):
    w = inputs.by_name(kind, n, 3000 + n)
    if w.sum() == 0:
        w[0] = 1.0
    cfg = wrs.config()
    prob, alias, inf, greedy = build_plus(w, 1, cfg)
    assert inf["status"] == wrs.OK
    assert inf["W"] == oracle.exact_sum(w)
    assert np.all((prob >= 0) & (prob <= 1))
    assert np.all(alias < n)
    assert mass_err(w, prob, alias) <= MASS_TOL
    _, _, g_orc = oracle.psa_plus(w, cfg.section_size, TILE, 1)
    assert greedy == g_orc, (greedy, g_orc)
    if n >= 4 * TILE:
        assert greedy > n // 2   # most of the table is packed greedily


@pytest.mark.parametrize("m", [8, 64, 200])
def test_plus_min_items(m):
    n = 200003
    w = inputs.by_name("gamma", n, 41)
    prob, alias, inf, greedy = build_plus(w, m)
    assert inf["status"] == wrs.OK
    assert mass_err(w, prob, alias) <= MASS_TOL
    _, _, g_orc = oracle.psa_plus(w, wrs.config().section_size, TILE, m)
    assert greedy == g_orc, (greedy, g_orc)


@pytest.mark.parametrize("kind", KINDS)
def test_plus_without_eligible_chunk_is_psa(kind):
    # min_items above the chunk size: every item goes to PSA in index order
    n = 70001
    w = inputs.by_name(kind, n, 51)
    if w.sum() == 0:
        w[0] = 1.0
    prob, alias, inf, greedy = build_plus(w, TILE + 1)
    assert greedy == 0
    b = wrs.Builder(n, wrs.config())
    rows = b.build(torch.from_numpy(w).cuda())
    torch.cuda.synchronize()
    p2, a2 = wrs.rows_to_numpy(rows)
    assert np.array_equal(prob.view(np.uint32), p2.view(np.uint32))
    assert np.array_equal(alias, a2)
    ref = wrs.parse_info(b.info)
    for k in ("status", "W", "avg", "nl", "nh", "Q", "light_max", "sections"):
        assert inf[k] == ref[k], k


def test_plus_unaligned_and_deterministic():
    # weights one float past a 16-byte boundary take the scalar-load path
    n = 300007
    w = inputs.by_name("exponential", n, 61)
    p0, a0, i0, g0 = build_plus(w, 1)
    p1, a1, i1, g1 = build_plus(w, 1, offset=1)
    p2, a2, _, g2 = build_plus(w, 1)
    assert i0["status"] == i1["status"] == wrs.OK
    assert g0 == g1 == g2
    for p, a in ((p1, a1), (p2, a2)):
        assert np.array_equal(p0.view(np.uint32), p.view(np.uint32))
        assert np.array_equal(a0, a)


def test_plus_degenerate_weights():
    # equal weights: every item is light (w <= avg), no chunk is eligible
    n = 5000
    w = np.full(n, 0.75, np.float32)
    prob, alias, inf, greedy = build_plus(w, 1)
    assert inf["status"] == wrs.OK and greedy == 0
    assert mass_err(w, prob, alias) <= MASS_TOL
    # one heavy per chunk, its excess exactly the chunk's whole deficit: the
    # heavy falls to the average after the last light and, with no next heavy
    # in the chunk, goes to the rest with weight avg (an exact tie on both sides)
    w = np.ones(4 * TILE, np.float32)
    w[::TILE] = 100.0
    prob, alias, inf, greedy = build_plus(w, 1)
    assert inf["status"] == wrs.OK
    assert mass_err(w, prob, alias) <= MASS_TOL
    _, _, g_orc = oracle.psa_plus(w, wrs.config().section_size, TILE, 1)
    assert greedy == g_orc == 4 * (TILE - 1)


@pytest.mark.parametrize("bad,status", [("zero", wrs.EZEROSUM), ("nan", wrs.ENONFINITE),
                                        ("inf", wrs.ENONFINITE), ("neg", wrs.EINVAL)])
def test_plus_status(bad, status):
    n = 4097
    w = np.zeros(n, np.float32) if bad == "zero" else inputs.by_name("uniform", n, 71)
    if bad == "nan":
        w[1234] = np.nan
    elif bad == "inf":
        w[7] = np.inf
    elif bad == "neg":
        w[4000] = -1.0
    _, _, inf, greedy = build_plus(w, 1)
    assert inf["status"] == status
    assert greedy == 0


def test_plus_large():
    n = (1 << 22) + 77
    w = inputs.by_name("gamma", n, 81)
    prob, alias, inf, greedy = build_plus(w, 1)
    assert inf["status"] == wrs.OK
    assert mass_err(w, prob, alias) <= MASS_TOL
    _, _, g_orc = oracle.psa_plus(w, wrs.config().section_size, TILE, 1)
    assert greedy == g_orc, (greedy, g_orc)


@pytest.mark.parametrize("kind,pos", [("uniform", 777), ("exponential", 1000)])
def test_plus_dominant_heavy(kind, pos):
    # one item holding half the weight: its excess key is past the 64-bit cap
    # (E' >= 2^77), so the carried weight comes from the exact sums (with
    # exponential weights other heavies of its chunk close before it)
    n = (1 << 20) + 5
    w = inputs.by_name(kind, n, 91)
    w[pos] = np.float32(w.astype(np.float64).sum())
    prob, alias, inf, greedy = build_plus(w, 1)
    assert inf["status"] == wrs.OK
    assert mass_err(w, prob, alias) <= MASS_TOL
    _, _, g_orc = oracle.psa_plus(w, wrs.config().section_size, TILE, 1)
    assert greedy == g_orc, (greedy, g_orc)


@pytest.mark.parametrize("section,method", [(256, 0), (8192, 0), (1024, 1)])
def test_plus_config(section, method):
    # the leftovers' PSA takes the section size and split method of cfg
    n = 250007
    w = inputs.by_name("exponential", n, 101)
    cfg = wrs.config(section, method)
    prob, alias, inf, greedy = build_plus(w, 1, cfg)
    assert inf["status"] == wrs.OK
    assert mass_err(w, prob, alias) <= MASS_TOL
    _, _, g_orc = oracle.psa_plus(w, section, TILE, 1)
    assert greedy == g_orc, (greedy, g_orc)
    # the greedy step does not depend on cfg: same greedy rows as the default
    p0, a0, _, g0 = build_plus(w, 1)
    assert g0 == greedy
