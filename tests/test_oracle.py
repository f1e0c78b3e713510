"""Pins for the CPU oracle (no GPU).

The oracle is only trusted after it agrees with things other than itself:
hand-worked fixtures (tests/golden), closed forms of the alias table
(Sec. 2.2), brute force on tiny inputs, exact rational arithmetic, library
routines that compute the same definition (math.fsum, numpy.searchsorted,
Triton's interpreted Philox) and statistical laws of the sampler.
"""
from __future__ import annotations

import itertools
import math
import struct
from fractions import Fraction

import numpy as np
import pytest

import oracle
from golden_io import fractions, ints, read
from paper_2106_12270_gb300 import inputs


def f32_from_bits(hexes):
    return np.array([struct.unpack("<f", struct.pack("<I", int(h, 16)))[0]
                     for h in hexes], np.float32)


def exact_rational_sum(w) -> Fraction:
    return sum((Fraction(float(x)) for x in np.asarray(w, np.float32)), Fraction(0))


# --------------------------------------------------------------------------
# exact sum (Sec. 1 defines W; exact summation, rounded once, is our reading)
# --------------------------------------------------------------------------

def test_exact_sum_golden_rounding():
    g = read("exact_sum_rounding.txt")
    for key, spec in g.items():
        lhs, rhs = spec.split("->")
        w = f32_from_bits(lhs.split())
        got = oracle.exact_sum(w)
        want = struct.unpack("<d", struct.pack("<Q", int(rhs.strip(), 16)))[0]
        assert struct.pack("<d", got) == struct.pack("<d", want), key


@pytest.mark.parametrize("kind", ["uniform", "zipf", "exponential", "gamma"])
def test_exact_sum_matches_fsum(kind):
    for seed in range(4):
        w = inputs.by_name(kind, 20000 + 37 * seed, seed)
        assert oracle.exact_sum(w) == math.fsum(w.astype(np.float64))


def test_exact_sum_matches_rationals_wide_range():
    rng = np.random.default_rng(11)
    for _ in range(30):
        n = int(rng.integers(1, 60))
        e = rng.integers(-149, 127, n)
        m = rng.random(n) + 0.5
        w = np.ldexp(m, e).astype(np.float32)
        w[~np.isfinite(w)] = 1.0
        want = float(exact_rational_sum(w))
        assert oracle.exact_sum(w) == want


def test_exact_sum_rejects_bad_weights():
    with pytest.raises(oracle.OracleError) as e:
        oracle.exact_sum(np.array([1.0, -2.0], np.float32))
    assert e.value.code == oracle.EINVAL
    for bad in (np.nan, np.inf):
        with pytest.raises(oracle.OracleError) as e:
            oracle.exact_sum(np.array([1.0, bad], np.float32))
        assert e.value.code == oracle.ENONFINITE


# --------------------------------------------------------------------------
# classification (Sec. 2.2: light iff w_i <= W/N; lists in index order)
# --------------------------------------------------------------------------

def test_classify_worked_example():
    g = read("alias_worked_1807.txt")
    w = np.array(ints(g["weights"]), np.float32)
    W = oracle.exact_sum(w)
    assert W == int(g["W"])
    l, h = oracle.classify(w, W / w.size)
    assert l.tolist() == ints(g["light"])
    assert h.tolist() == ints(g["heavy"])


def test_classify_tie_is_light():
    w = np.full(17, 0.3, np.float32)
    l, h = oracle.classify(w, oracle.exact_sum(w) / w.size)
    assert len(l) == 17 and len(h) == 0


def test_classify_partition_properties():
    w = inputs.exponential(5000, 4)
    avg = oracle.exact_sum(w) / w.size
    l, h = oracle.classify(w, avg)
    assert np.all(np.diff(l.astype(np.int64)) > 0) and np.all(np.diff(h.astype(np.int64)) > 0)
    assert sorted(np.concatenate([l, h]).tolist()) == list(range(w.size))
    assert np.all(w[l].astype(np.float64) <= avg) and np.all(w[h].astype(np.float64) > avg)


# --------------------------------------------------------------------------
# Vose (Sec. 2.2)
# --------------------------------------------------------------------------

def _check_golden_table(name, build, rows=False):
    g = read(name)
    w = np.array(ints(g["weights"]), np.float32)
    t = build(w)
    assert t["nl"] == int(g["nl"]) and t["nh"] == int(g["nh"])
    want_mass = fractions(g["mass"])
    got = oracle.mass(t["prob"], t["alias"])
    assert [Fraction(float(x)) for x in got] == want_mass
    if rows and "sweep_prob" in g:
        assert [Fraction(float(x)) for x in t["prob"]] == fractions(g["sweep_prob"])
        assert t["alias"].tolist() == ints(g["sweep_alias"])


@pytest.mark.parametrize("name", ["alias_worked_1807.txt", "alias_worked_3311.txt",
                                  "alias_worked_1124.txt"])
def test_vose_golden(name):
    _check_golden_table(name, oracle.vose)


@pytest.mark.parametrize("name", ["alias_worked_1807.txt", "alias_worked_3311.txt",
                                  "alias_worked_1124.txt"])
@pytest.mark.parametrize("section", [1, 2, 3, 4])
def test_psa_golden(name, section):
    _check_golden_table(name, lambda w: oracle.psa(w, section), rows=True)


def test_psa_golden_splits():
    g = read("alias_worked_1807.txt")
    w = np.array(ints(g["weights"]), np.float32)
    t = oracle.psa(w, 1)
    assert t["split_i"].tolist() == ints(g["split_i"])
    assert t["split_j"].tolist() == ints(g["split_j"])
    assert [Fraction(float(x)) for x in t["spill"]] == fractions(g["spill"])


def test_vose_closed_forms():
    t = oracle.vose(np.array([2.5], np.float32))
    assert t["prob"].tolist() == [1.0] and t["alias"].tolist() == [0]
    t = oracle.vose(np.full(9, 0.7, np.float32))
    assert np.all(t["prob"] == 1.0) and t["nh"] == 0
    t = oracle.vose(np.array([0, 0, 5, 0], np.float32))
    assert t["prob"][2] == 1.0
    for i in (0, 1, 3):
        assert t["prob"][i] == 0.0 and t["alias"][i] == 2
    for a, b in [(1.0, 3.0), (0.25, 0.5), (0.0, 1.0), (2.0, 7.0)]:
        t = oracle.vose(np.array([a, b], np.float32))
        assert t["prob"][0] == pytest.approx(2 * a / (a + b), abs=1e-15)
        assert t["alias"][0] == 1 and t["prob"][1] == 1.0


def _all_small_vectors():
    grid = [0.0, 0.5, 1.0, 2.0, 3.0]
    for n in range(1, 5):
        for v in itertools.product(grid, repeat=n):
            if any(v):
                yield np.array(v, np.float32)


def test_vose_and_psa_brute_force_tiny():
    """Every weight vector over a small grid, N <= 4: the mass each table
    gives every item equals N*w_i/W, checked in exact rationals up to FP64
    round-off of the kept shares."""
    for w in _all_small_vectors():
        W = exact_rational_sum(w)
        n = w.size
        want = [Fraction(n) * Fraction(float(x)) / W for x in w]
        for t in [oracle.vose(w)] + [oracle.psa(w, s) for s in range(1, n + 1)]:
            assert np.all((t["prob"] >= 0) & (t["prob"] <= 1))
            assert np.all(t["alias"] < n)
            got = oracle.mass(t["prob"], t["alias"])
            for g, e in zip(got, want):
                assert abs(Fraction(float(g)) - e) <= Fraction(1, 2**40)


@pytest.mark.parametrize("kind", ["uniform", "zipf", "exponential", "gamma"])
def test_vose_mass_and_invariants(kind):
    w = inputs.by_name(kind, 30000, 5)
    t = oracle.vose(w)
    assert oracle.mass_error(t["prob"], t["alias"], w, t["W"]) < 1e-9
    m = oracle.mass(t["prob"], t["alias"])
    assert abs(m.sum() - w.size) < 1e-6
    assert np.all(m[w == 0] == 0.0)


# --------------------------------------------------------------------------
# PSA splits and pack (Sec. 2.2, Sec. 4.1, Sec. 4.2)
# --------------------------------------------------------------------------

def _split_brute(sl, sh, avg, k):
    nl, nh = len(sl) - 1, len(sh) - 1
    lo, hi = max(0, k - nh), min(k, nl)
    for i in range(lo, hi + 1):
        if i == hi or sl[i] + sh[k - i] - k * avg <= 0.0:
            return i
    raise AssertionError


@pytest.mark.parametrize("kind", ["uniform", "zipf", "exponential", "gamma"])
def test_split_binary_and_pary_equal_brute_force(kind):
    for seed, n in [(1, 300), (2, 1000), (3, 77)]:
        w = inputs.by_name(kind, n, seed)
        W = oracle.exact_sum(w)
        avg = W / n
        l, h = oracle.classify(w, avg)
        sl, sh = oracle.prefix(w, l), oracle.prefix(w, h)
        ks = np.arange(0, n + 1, dtype=np.uint64)
        want = [_split_brute(sl, sh, avg, int(k)) for k in ks]
        i, j, sp = oracle.split_binary(sl, sh, avg, ks)
        assert i.tolist() == want
        assert (i + j).tolist() == ks.tolist()
        for p in (2, 3, 8, 32, 256):
            ip, jp, spp = oracle.split_pary(sl, sh, avg, ks, p)
            assert ip.tolist() == want
            assert np.array_equal(spp, sp)


def test_pary_search_equals_searchsorted():
    rng = np.random.default_rng(9)
    for _ in range(50):
        n = int(rng.integers(0, 3000))
        lst = np.sort(rng.integers(0, 500, n).astype(np.float64))
        keys = np.sort(rng.integers(-5, 505, int(rng.integers(1, 700))).astype(np.float64))
        want = np.searchsorted(lst, keys, side="right")
        for p in (2, 4, 32, 128):
            assert np.array_equal(oracle.pary_search(lst, keys, p), want)


@pytest.mark.parametrize("kind", ["uniform", "zipf", "exponential", "gamma"])
def test_psa_sections_reproduce_one_sweep(kind):
    """Splitting must land on the states a single sweep passes through:
    every section size gives the same table as one section (S = N)."""
    n = 4000
    w = inputs.by_name(kind, n, 12)
    whole = oracle.psa(w, n)
    for S in (1, 7, 64, 1000):
        t = oracle.psa(w, S)
        assert np.array_equal(t["alias"], whole["alias"])
        assert np.max(np.abs(t["prob"] - whole["prob"])) < 1e-9
        t2 = oracle.psa(w, S, pary_p=32)
        assert np.array_equal(t2["alias"], t["alias"])


@pytest.mark.parametrize("kind", ["uniform", "zipf", "exponential", "gamma"])
def test_psa_mass_matches_vose(kind):
    w = inputs.by_name(kind, 50000, 21)
    v = oracle.vose(w)
    t = oracle.psa(w, 512)
    assert t["nl"] == v["nl"] and t["nh"] == v["nh"]
    assert oracle.mass_error(t["prob"], t["alias"], w, v["W"]) < 1e-9
    mv = oracle.mass(v["prob"], v["alias"])
    mt = oracle.mass(t["prob"], t["alias"])
    assert np.max(np.abs(mv - mt) / np.maximum(1.0, mv)) < 1e-9


def test_split_invariant_each_section_closes_its_buckets():
    w = inputs.zipf_permuted(20000, 8)
    S = 333
    t = oracle.psa(w, S)
    k = np.minimum(np.arange(len(t["split_i"]), dtype=np.int64) * S, w.size)
    assert np.array_equal(t["split_i"].astype(np.int64) + t["split_j"].astype(np.int64), k)
    assert np.all(np.diff(t["split_i"].astype(np.int64)) >= 0)
    assert np.all(np.diff(t["split_j"].astype(np.int64)) >= 0)


# --------------------------------------------------------------------------
# Philox-4x32-10 (Salmon et al., SC'11) against Triton's interpreted Philox
# --------------------------------------------------------------------------

def test_philox_matches_triton_interpreter():
    import os
    os.environ.setdefault("TRITON_INTERPRET", "1")
    if os.environ.get("TRITON_INTERPRET") != "1":
        pytest.skip("Triton interpreter not enabled")
    torch = pytest.importorskip("torch")
    triton = pytest.importorskip("triton")
    tl = pytest.importorskip("triton.language")

    @triton.jit
    def kern(out, c0p, c1p, c2p, c3p, seed, N: tl.constexpr):
        offs = tl.arange(0, N)
        c0 = tl.load(c0p + offs).to(tl.uint32, bitcast=True)
        c1 = tl.load(c1p + offs).to(tl.uint32, bitcast=True)
        c2 = tl.load(c2p + offs).to(tl.uint32, bitcast=True)
        c3 = tl.load(c3p + offs).to(tl.uint32, bitcast=True)
        a, b, c, d = tl.philox(seed, c0, c1, c2, c3, 10)
        tl.store(out + offs * 4 + 0, a.to(tl.int32, bitcast=True))
        tl.store(out + offs * 4 + 1, b.to(tl.int32, bitcast=True))
        tl.store(out + offs * 4 + 2, c.to(tl.int32, bitcast=True))
        tl.store(out + offs * 4 + 3, d.to(tl.int32, bitcast=True))

    rng = np.random.default_rng(3)
    N = 16
    for seed in (0, 1, 0x0123456789ABCDEF, 2**64 - 1):
        ctr = rng.integers(0, 2**32, (4, N), dtype=np.uint64).astype(np.uint32)
        ctr[:, 0] = 0
        ctr[:, 1] = 0xFFFFFFFF
        cts = [torch.from_numpy(ctr[r].view(np.int32).copy()) for r in range(4)]
        out = torch.zeros(4 * N, dtype=torch.int32)
        kern[(1,)](out, *cts, seed, N)
        got = out.numpy().view(np.uint32).reshape(N, 4)
        for q in range(N):
            key = [seed & 0xFFFFFFFF, seed >> 32]
            want = oracle.philox(ctr[:, q], key)
            assert got[q].tolist() == want.tolist(), (seed, q)


def test_philox_output_is_uniform():
    from scipy import stats
    words = np.concatenate([oracle.philox([c, 0, 7, 0], [5, 6]) for c in range(4000)])
    counts = np.bincount((words >> 24).astype(np.int64), minlength=256)
    assert stats.chisquare(counts).pvalue > 1e-4


# --------------------------------------------------------------------------
# Sampling (Sec. 2.2, Sec. 5)
# --------------------------------------------------------------------------

def _gof(samples, n, probs):
    from scipy import stats
    counts = np.bincount(samples.astype(np.int64), minlength=n)
    probs = np.asarray(probs, np.float64)
    exp = probs / probs.sum() * samples.size
    keep = exp > 0
    assert counts[~keep].sum() == 0
    return stats.chisquare(counts[keep], exp[keep]).pvalue


def test_naive_sampler_goodness_of_fit():
    w = np.array([1, 8, 0, 7, 3, 0.5, 12, 2], np.float32)
    t = oracle.vose(w)
    s = oracle.sample_naive(t["prob"].astype(np.float32), t["alias"], 0, 400000, seed=2)
    assert _gof(s, w.size, w / w.sum()) > 1e-3


def test_naive_sampler_edge_rows():
    n = 1 << 10
    prob = np.ones(n, np.float32)
    alias = np.zeros(n, np.uint32)
    s = oracle.sample_naive(prob, alias, 0, 1000, seed=9)
    # prob 1 keeps the row: the row is the top 10 bits of the 64-bit draw
    for q in range(0, 1000, 97):
        x = oracle.philox([q // 2, 0, 0, 0], [9, 0])
        u = (int(x[0]) << 32 | int(x[1])) if q % 2 == 0 else (int(x[2]) << 32 | int(x[3]))
        assert s[q] == u >> 54
    s0 = oracle.sample_naive(np.zeros(n, np.float32), alias, 0, 1000, seed=9)
    assert np.all(s0 == 0)  # prob 0 always takes the alias


def test_naive_sampler_offsets_are_consistent():
    w = inputs.uniform(500, 1)
    t = oracle.vose(w)
    p32 = t["prob"].astype(np.float32)
    full = oracle.sample_naive(p32, t["alias"], 0, 1001, seed=77, stream_lo=3)
    part = oracle.sample_naive(p32, t["alias"], 333, 400, seed=77, stream_lo=3)
    assert np.array_equal(full[333:733], part)


def test_sectioned_sampler_stays_in_sections_and_fits():
    w = inputs.exponential(1000, 3)
    t = oracle.vose(w)
    p32 = t["prob"].astype(np.float32)
    nsec = 7
    bounds = [(s * w.size) // nsec for s in range(nsec + 1)]
    counts = np.array([(bounds[s + 1] - bounds[s]) * 300 for s in range(nsec)], np.uint64)
    out = oracle.sample_sectioned(p32, t["alias"], counts, seed=4, tag=1)
    pos = 0
    for s in range(nsec):
        seg = out[pos: pos + int(counts[s])]
        pos += int(counts[s])
        rows_ok = (seg >= bounds[s]) & (seg < bounds[s + 1])
        alias_ok = np.isin(seg, t["alias"][bounds[s]:bounds[s + 1]])
        assert np.all(rows_ok | alias_ok)
    # counts proportional to section sizes make the whole stream exact in law
    assert _gof(out, w.size, w.astype(np.float64) / w.astype(np.float64).sum()) > 1e-3


# --------------------------------------------------------------------------
# Precision study: the PSA's prefix arithmetic in FP64, paired FP32
# (compensated summation) and plain FP32
# --------------------------------------------------------------------------

@pytest.mark.parametrize("kind", ["uniform", "zipf", "exponential"])
def test_precision_study_prefix_arithmetic(kind):
    """FP64 working precision reproduces orc_psa bit for bit; FP64 and paired
    FP32 (about 48 bits) meet the 1e-5 mass bound for an FP32-stored table;
    plain FP32 prefix sums miss it by orders of magnitude at 2e6 items."""
    n = 2_000_000
    w = inputs.by_name(kind, n, 11)
    W = oracle.exact_sum(w)
    ref = oracle.psa(w, 1024)
    errs = []
    for prec in (oracle.PREC_FP64, oracle.PREC_FP32_PAIR, oracle.PREC_FP32):
        prob, alias = oracle.psa_prec(w, 1024, prec)
        if prec == oracle.PREC_FP64:
            assert np.array_equal(prob, ref["prob"]) and np.array_equal(alias, ref["alias"])
        p32 = prob.astype(np.float32).astype(np.float64)
        errs.append(oracle.mass_error(p32, alias, w, W))
    assert errs[0] <= 1e-6 and errs[1] <= 1e-5 and errs[2] > 1e-3, errs


# --------------------------------------------------------------------------
# PSA+ (Sec. 4 "PSA+"): greedy packing per tile, then PSA on the rest
# --------------------------------------------------------------------------

def test_psa_plus_golden():
    g = read("psa_plus_worked_1313.txt")
    w = np.array([float(x) for x in g["weights"].split()], np.float32)
    prob, alias, greedy = oracle.psa_plus(w, 1024, int(g["tile"]), int(g["min_items"]))
    assert greedy == int(g["greedy"])
    assert [Fraction(p).limit_denominator(64) for p in prob] == fractions(g["prob"])
    assert alias.tolist() == ints(g["alias"])
    assert [Fraction(m).limit_denominator(64) for m in oracle.mass(prob, alias)] == \
        fractions(g["mass"])


@pytest.mark.parametrize("kind", ["uniform", "zipf", "exponential", "gamma"])
def test_psa_plus_without_greedy_step_is_psa(kind):
    """With no tile eligible for greedy packing, PSA+ is PSA (binary split),
    bit for bit."""
    w = inputs.by_name(kind, 20011, 3)
    ref = oracle.psa(w, 1024)
    prob, alias, greedy = oracle.psa_plus(w, 1024, 4096, 10**9)
    assert greedy == 0
    assert np.array_equal(prob, ref["prob"]) and np.array_equal(alias, ref["alias"])


def test_psa_plus_brute_force_masses():
    """Every weight vector over {0, 1/2, 1, 2, 3}^N, N <= 4, every tile size
    and threshold: each item's reconstructed mass is N w_i / W."""
    vals = [0.0, 0.5, 1.0, 2.0, 3.0]
    for N in range(1, 5):
        for ws in itertools.product(vals, repeat=N):
            w = np.array(ws, np.float32)
            if w.sum() == 0:
                continue
            W = float(w.astype(np.float64).sum())
            want = w.astype(np.float64) * N / W
            for T in sorted({1, 2, 3, N}):
                for m in (1, 2):
                    for S in (1, 2, 1024):
                        prob, alias, _ = oracle.psa_plus(w, S, T, m)
                        assert np.all((prob >= 0) & (prob <= 1)) and np.all(alias < N)
                        got = oracle.mass(prob, alias)
                        assert np.allclose(got, want, rtol=0, atol=1e-12), (ws, T, m, S)


@pytest.mark.parametrize("kind", ["uniform", "zipf", "exponential", "gamma"])
@pytest.mark.parametrize("tile, m", [(64, 1), (512, 8), (4096, 1)])
def test_psa_plus_masses_random(kind, tile, m):
    w = inputs.by_name(kind, 100_003, 9)
    W = oracle.exact_sum(w)
    prob, alias, greedy = oracle.psa_plus(w, 1024, tile, m)
    assert 0 < greedy <= w.size
    assert np.all((prob >= 0) & (prob <= 1)) and np.all(alias < w.size)
    e = oracle.expected_mass(w, W)
    assert np.max(np.abs(oracle.mass(prob, alias) - e) / np.maximum(1.0, e)) <= 1e-9


def test_psa_plus_greedy_share_uniform():
    """Sec. 6 (PSA+): with uniform random weights the greedy step finishes
    around 90% of the items on GPU-sized tiles."""
    w = inputs.uniform(1_000_000, 1)
    _, _, greedy = oracle.psa_plus(w, 1024, 512, 1)
    assert greedy / w.size >= 0.85


def test_near_tie_check_flags_a_planted_alias():
    """The parity tests' near-tie check (gpu_util.alias_differences_at_ties)
    accepts an identical table and flags a light row whose alias names a
    heavy three places away from the sweep's choice (no tie there)."""
    from fractions import Fraction

    from gpu_util import alias_differences_at_ties, fixed_q_exact
    w = inputs.exponential(5000, 3)
    n = w.size
    t = oracle.psa(w, 1024)
    W = oracle.exact_sum(w)
    Wx = sum((Fraction(float(x)) for x in w), Fraction(0))
    S = 0
    while Wx * Fraction(2) ** S >= 2**62:
        S -= 1
    while Wx * Fraction(2) ** S < 2**61:
        S += 1
    q = fixed_q_exact(w, S)
    exact = [int((Fraction(float(x)) * Fraction(2) ** S + Fraction(1, 2)) // 1) for x in w]
    assert list(map(int, q)) == exact
    info = {"scale": S, "Q": sum(exact)}
    assert alias_differences_at_ties(w, info, t["alias"], t["alias"]) == (0, [])
    l, h = oracle.classify(w, W / n)
    bad = t["alias"].copy()
    y = int(np.searchsorted(h, bad[l[100]]))
    bad[l[100]] = h[min(len(h) - 1, y + 3)]
    assert alias_differences_at_ties(w, info, bad, t["alias"]) == (1, [int(l[100])])
