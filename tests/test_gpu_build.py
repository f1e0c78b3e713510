"""Parity of the CUDA construction path with the CPU oracle (GPU required).

Every step runs through the C ABI (libwrs.so).  Tolerances:
* total weight W, light/heavy counts, the l/h lists: bit-exact;
* prefix-sum checkpoints: within N (i + N) / Q buckets of the exact rational
  prefix sums -- the fixed point rounds each weight to 2^-S (half a unit),
  Q = sum of the rounded weights >= 2^61;
* splits: equal to the oracle's PSA splits (FP64 binary search);
* table: |mass_i - N w_i/W| <= 1e-5 max(1, N w_i/W) (the stated bound for
  FP32 tables) and agreement with the oracle's PSA rows.
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np
import pytest
import torch

import oracle
import paper_2106_12270_gb300 as wrs
from gpu_util import Built, alias_differences_at_ties, exact_prefix
from paper_2106_12270_gb300 import inputs

pytestmark = pytest.mark.gpu

MASS_TOL = 1e-5
KINDS = ["uniform", "zipf", "exponential", "gamma"]
# sizes spanning several partition tiles (4096 items) and sections, ragged tails
SIZES = [1, 2, 3, 31, 32, 33, 255, 4095, 4096, 4097, 12289, 100003]


def mass_ok(b: Built, W: float):
    e = oracle.expected_mass(b.w, W)
    m = oracle.mass(b.prob.astype(np.float64), b.alias)
    err = np.abs(m - e) / np.maximum(1.0, e)
    return float(err.max()) if err.size else 0.0


def check_table(b: Built):
    assert b.info["status"] == wrs.OK
    assert np.all((b.prob >= 0) & (b.prob <= 1))
    assert np.all(b.alias < b.n)
    W = oracle.exact_sum(b.w)
    assert mass_ok(b, W) <= MASS_TOL


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("n", SIZES)
def test_build_matches_oracle(kind, n):
    w = inputs.by_name(kind, n, 1000 + n)
    if w.sum() == 0:
        w[0] = 1.0
    b = Built(w)
    W = oracle.exact_sum(w)
    # a1: exact total, bit for bit
    assert b.info["W"] == W
    assert b.info["avg"] == W / n
    # a2: classification and stable partition, bit for bit
    l, h = oracle.classify(w, W / n)
    assert (b.info["nl"], b.info["nh"]) == (len(l), len(h))
    li, lw, hi, hw = b.lists()
    assert np.array_equal(li, l) and np.array_equal(hi, h)
    assert np.array_equal(lw, w[l]) and np.array_equal(hw, w[h])
    check_table(b)
    # a5 vs the oracle's PSA sweep with the same sections
    t = oracle.psa(w, b.cfg.section_size)
    same = b.alias == t["alias"]
    # only near-ties of the FP64 sweep may differ (none do on these inputs)
    _, not_ties = alias_differences_at_ties(w, b.info, b.alias, t["alias"])
    assert not not_ties, not_ties[:10]
    assert np.max(np.abs(b.prob[same] - t["prob"][same])) < 1e-6


@pytest.mark.parametrize("kind", KINDS)
def test_prefix_checkpoints_exact(kind):
    n = 20011
    w = inputs.by_name(kind, n, 7)
    b = Built(w)
    Wx = sum((Fraction(float(x)) for x in w), Fraction(0))
    Q = b.info["Q"]
    li, _, hi, _ = b.lists()
    for which, lst, sign in (("ckl", li, 1), ("ckh", hi, -1)):
        ck = b.checkpoints(which)
        ex = exact_prefix(w, lst, 32)
        assert len(ck) == len(ex)
        for c, (sig_q, sig) in enumerate(zip(ck, ex)):
            i = 32 * c
            # D'(i)/Q = i - N sigma_q/Q (lights), E'(i)/Q = N sigma_q/Q - i (heavies);
            # exact: i - sigma N/W and sigma N/W - i
            got = sign * Fraction(i * Q - n * sig_q, Q)
            want = sign * (i - sig * n / Wx)
            assert abs(got - want) <= Fraction(n * (i + n), Q), (which, c)


def fixed_point_q(w, S):
    """q_i = floor(w_i 2^S + 1/2): each weight rounded to the fixed point,
    halves up, in exact rational arithmetic."""
    scale = Fraction(2) ** S
    half = Fraction(1, 2)
    return [int((Fraction(float(x)) * scale + half) // 1) for x in w]


@pytest.mark.parametrize("kind", KINDS)
def test_fixed_point_exact(kind):
    """The fixed point bit for bit: the scale puts W 2^S in [2^61, 2^62),
    Q is the sum of the rounded weights, and every checkpoint is the exact sum
    of the clamped q (lights at most floor(Q/N), heavies at least that + 1)."""
    n = 20011
    w = inputs.by_name(kind, n, 17)
    b = Built(w)
    S = b.info["scale"]
    Wx = sum((Fraction(float(x)) for x in w), Fraction(0))
    assert 2**61 <= Wx * Fraction(2) ** S < 2**62
    q = fixed_point_q(w, S)
    Q = sum(q)
    assert b.info["Q"] == Q
    Qn = Q // n
    li, _, hi, _ = b.lists()
    for which, lst, clamp in (("ckl", li, lambda v: min(v, Qn)),
                              ("ckh", hi, lambda v: max(v, Qn + 1))):
        ck = b.checkpoints(which)
        acc, want = 0, []
        for a, idx in enumerate(lst):
            if a % 32 == 0:
                want.append(acc)
            acc += clamp(q[int(idx)])
        if len(lst) % 32 == 0:
            want.append(acc)
        assert ck == want, which


def _near_threshold(kind: str, n: int) -> np.ndarray:
    r = np.random.default_rng(23)
    if kind == "near":       # every weight within 2^-17 of 1
        return (1.0 + r.integers(-64, 64, n) * 2.0**-23).astype(np.float32)
    if kind == "equal":
        return np.full(n, 0.37, np.float32)
    w = r.exponential(1.0, n).astype(np.float32)   # Exp(1) with 1% at the float mean
    w[r.random(n) < 0.01] = np.float32(w.astype(np.float64).mean())
    return w


@pytest.mark.parametrize("kind", ["near", "equal", "exp_at_mean"])
def test_fixed_point_exact_near_threshold(kind):
    """Weights at or next to the light threshold: the partition's per-chunk
    test sends these chunks through the clamped pass; its checkpoints must
    still be the exact clamped sums."""
    n = 20011
    w = _near_threshold(kind, n)
    b = Built(w)
    S = b.info["scale"]
    q = fixed_point_q(w, S)
    Q = sum(q)
    assert b.info["Q"] == Q
    Qn = Q // n
    l, h = oracle.classify(w, oracle.exact_sum(w) / n)
    assert (b.info["nl"], b.info["nh"]) == (len(l), len(h))
    li, _, hi, _ = b.lists()
    for which, lst, clamp in (("ckl", li, lambda v: min(v, Qn)),
                              ("ckh", hi, lambda v: max(v, Qn + 1))):
        ck = b.checkpoints(which)
        acc, want = 0, []
        for a, idx in enumerate(lst):
            if a % 32 == 0:
                want.append(acc)
            acc += clamp(q[int(idx)])
        if len(lst) % 32 == 0:
            want.append(acc)
        assert ck == want, which
    check_table(b)


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("section", [256, 1024, 4096])
@pytest.mark.parametrize("method", [wrs.SPLIT_PARY, wrs.SPLIT_BINARY])
def test_splits_match_oracle(kind, section, method):
    n = 300007
    w = inputs.by_name(kind, n, 3)
    b = Built(w, wrs.config(section, method))
    i, j, D, E = b.splits()
    t = oracle.psa(w, section)
    assert np.array_equal(i, t["split_i"].astype(np.int64))
    assert np.array_equal(j, t["split_j"].astype(np.int64))
    check_table(b)


def test_split_methods_bit_identical():
    n = 1 << 20
    w = inputs.zipf_permuted(n, 5)
    a = Built(w, wrs.config(1024, wrs.SPLIT_PARY))
    c = Built(w, wrs.config(1024, wrs.SPLIT_BINARY))
    assert a.splits()[0].tolist() == c.splits()[0].tolist()
    assert torch.equal(a.rows_t, c.rows_t)


@pytest.mark.parametrize("kind,n", [("exponential", 77777), ("gamma", 3_000_001)])
def test_steps_equal_full_build(kind, n):
    # the one-call build chains its later kernels as programmatic dependents;
    # the step calls run every kernel after its predecessor has finished
    w = inputs.by_name(kind, n, 2)
    a = Built(w)
    s = Built(w, steps=True)
    assert torch.equal(a.rows_t, s.rows_t)
    assert a.info == s.info


def test_unaligned_weights_pointer():
    w = inputs.uniform(50001, 9)
    big = torch.from_numpy(np.concatenate([[0.0], w]).astype(np.float32)).cuda()
    b = Built(w, w_tensor=big[1:])
    a = Built(w)
    assert torch.equal(a.rows_t, b.rows_t)


@pytest.mark.parametrize("section", [256, 8192])
def test_section_sizes(section):
    w = inputs.gamma(123457, 4)
    b = Built(w, wrs.config(section))
    check_table(b)


def test_deterministic_rebuild():
    w = inputs.zipf_permuted(1 << 18, 8)
    a = Built(w)
    c = Built(w)
    assert torch.equal(a.rows_t, c.rows_t)


# ---------------------------------------------------------------------------
# special cases of the method (Sec. 2.2)
# ---------------------------------------------------------------------------

def test_single_item():
    b = Built(np.array([3.5], np.float32))
    assert b.prob.tolist() == [1.0] and b.alias.tolist() == [0]


def test_all_equal_weights_are_light():
    b = Built(np.full(10007, 0.37, np.float32))
    assert b.info["nh"] == 0 and np.all(b.prob == 1.0)


def test_one_nonzero_weight():
    w = np.zeros(5000, np.float32)
    w[1234] = 2.0
    b = Built(w)
    check_table(b)
    assert b.info["nh"] == 1
    assert b.prob[1234] == 1.0
    others = np.arange(5000) != 1234
    assert np.all(b.prob[others] == 0.0) and np.all(b.alias[others] == 1234)


def test_two_items_closed_form():
    for a, c in [(1.0, 3.0), (0.25, 0.5), (0.0, 1.0), (2.0, 7.0)]:
        b = Built(np.array([a, c], np.float32))
        assert b.prob[0] == pytest.approx(2 * a / (a + c), abs=2e-7)
        assert b.alias[0] == 1 and b.prob[1] == 1.0


def test_wide_dynamic_range_and_subnormals():
    rng = np.random.default_rng(4)
    e = rng.integers(-149, 100, 40000)
    w = np.ldexp(rng.random(40000) + 0.5, e).astype(np.float32)
    w[~np.isfinite(w)] = 1e30
    w[::97] = 0.0
    w[5::101] = -0.0
    b = Built(w)
    assert b.info["W"] == oracle.exact_sum(w)
    check_table(b)


def test_weights_at_the_average():
    # many items exactly at W/N stay light (w_i <= W/N)
    w = np.concatenate([np.full(1000, 1.0), [0.5] * 10, [1.5] * 10]).astype(np.float32)
    b = Built(w)
    l, h = oracle.classify(w, oracle.exact_sum(w) / w.size)
    assert b.info["nl"] == len(l) and b.info["nh"] == len(h)
    check_table(b)


@pytest.mark.parametrize("bad, status", [(np.nan, wrs.ENONFINITE), (np.inf, wrs.ENONFINITE),
                                         (-1.0, wrs.EINVAL)])
def test_bad_weights_report_status(bad, status):
    w = inputs.uniform(9000, 1)
    w[4321] = bad
    b = Built(w)
    assert b.info["status"] == status


def test_all_zero_weights():
    b = Built(np.zeros(777, np.float32))
    assert b.info["status"] == wrs.EZEROSUM


def test_invalid_arguments_rejected_on_host():
    w = torch.ones(10, device="cuda")
    rows = torch.empty(10, dtype=torch.int64, device="cuda")
    info = torch.zeros(wrs.INFO_BYTES, dtype=torch.uint8, device="cuda")
    small = torch.empty(256, dtype=torch.uint8, device="cuda")
    with pytest.raises(wrs.WrsError) as e:
        wrs.build_rows(w, rows, small, info)
    assert e.value.status == wrs.EINVAL
    with pytest.raises(wrs.WrsError):
        wrs.build_workspace_bytes(10, wrs.config(300))  # not a multiple of 256


def test_total_weight_rounding_golden():
    """The device's exact sum rounds like IEEE binary64 ties-to-even: the
    hand-worked cases of tests/golden/exact_sum_rounding.txt."""
    import struct
    from golden_io import read
    for key, spec in read("exact_sum_rounding.txt").items():
        lhs, rhs = spec.split("->")
        w = np.array([struct.unpack("<f", struct.pack("<I", int(h, 16)))[0]
                      for h in lhs.split()], np.float32)
        want = struct.unpack("<d", struct.pack("<Q", int(rhs.strip(), 16)))[0]
        b = Built(w)
        if want == 0.0:
            assert b.info["status"] == wrs.EZEROSUM, key
        else:
            assert struct.pack("<d", b.info["W"]) == struct.pack("<d", want), key


def test_total_weight_wide_range_random():
    rng = np.random.default_rng(21)
    for trial in range(20):
        n = int(rng.integers(1, 5000))
        e = rng.integers(-149, 127, n)
        w = np.ldexp(rng.random(n) + 0.5, e).astype(np.float32)
        w[~np.isfinite(w)] = 3.0e38
        b = Built(w)
        assert b.info["W"] == oracle.exact_sum(w), trial
        l, h = oracle.classify(w, b.info["W"] / n)
        assert (b.info["nl"], b.info["nh"]) == (len(l), len(h))


@pytest.mark.parametrize("n", [1, 4097, 1_000_003])
def test_host_buffer_build_equals_device_build(n):
    """wrs_build_rows_host: weights and rows in (pinned) host memory, the
    copies on the stream; the same table as the device build."""
    w = inputs.by_name("zipf", n, 77)
    b = Built(w)
    cfg = wrs.config()
    ws = torch.empty(wrs.build_host_workspace_bytes(n, cfg), dtype=torch.uint8, device="cuda")
    w_pin = torch.from_numpy(w).pin_memory()
    rows_pin = torch.zeros(n, dtype=torch.int64).pin_memory()
    info_pin = torch.zeros(wrs.INFO_BYTES, dtype=torch.uint8).pin_memory()
    s = torch.cuda.Stream()
    wrs.build_rows_host(w_pin, rows_pin, ws, info_pin, cfg, s)
    s.synchronize()
    info = wrs.parse_info(info_pin)
    assert info["status"] == wrs.OK and info["W"] == b.info["W"]
    assert torch.equal(rows_pin, b.rows_t.cpu())
    # too small a workspace is refused before anything is enqueued
    with pytest.raises(wrs.WrsError):
        wrs.build_rows_host(w_pin, rows_pin, ws[: ws.numel() // 2], info_pin, cfg, s)
