"""CPU oracle for alias-table construction and sampling (test infrastructure).

This package is the independent, slow, FP64 reference the CUDA library is
checked against.  Only the test suite, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import it; the product library never does.

The arithmetic lives in ``oracle.c`` (plain C, compiled with gcc on first use
into ``oracle/_build/``).  This module only marshals numpy arrays.  Every
function cites the part of the paper (arXiv 2106.12270) it follows:

* ``exact_sum``       W = sum of the weights, exact, rounded once (Sec. 1).
* ``classify``        light iff w_i <= W/N, lists in index order (Sec. 2.2).
* ``vose``            Vose's sequential construction (Sec. 2.2).
* ``prefix``          prefix sums over a list of items (Sec. 2.2).
* ``split_binary``    PSA splits by binary search (Sec. 2.2, Sec. 4.1).
* ``split_pary``      PSA splits by partial p-ary search (Sec. 4.1, Alg. 1).
* ``pary_search``     Algorithm 1 on a sorted list (Sec. 4.1).
* ``psa``             PSA split + sweep-pack (Sec. 2.2, Sec. 4.2).
* ``psa_prec``        the same PSA with its prefix arithmetic rounded to FP64,
                      paired FP32 or plain FP32 (precision study).
* ``psa_plus``        PSA+ (Sec. 4): greedy packing per tile, PSA on the rest.
* ``mass``            reconstructed mass per item (Sec. 2.2).
* ``philox``          Philox-4x32-10 (Salmon et al., SC'11).
* ``sample_naive``    Walker sampling, integer form (Sec. 2.2, Sec. 5).
* ``sample_sectioned`` sampling inside sections given counts (Sec. 5).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

OK, EINVAL, EZEROSUM, ENONFINITE, ENOMEM = 0, -1, -2, -3, -4


class OracleError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"oracle {what} failed with code {code}")
        self.code = code


def build(force: bool = False) -> str:
    """Compile oracle.c into a shared library (gcc, -O2, no fast-math)."""
    os.makedirs(_BUILD, exist_ok=True)
    stale = (not os.path.exists(_LIB_PATH)
             or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC))
    if force or stale:
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.run(["gcc", "-std=c11", "-O2", "-fPIC", "-shared",
                        "-fno-fast-math", "-ffp-contract=off",
                        "-o", tmp, _SRC, "-lm"], check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            U64, U32, D = ctypes.c_uint64, ctypes.c_uint32, ctypes.c_double
            sigs = {
                "orc_exact_sum": [P, U64, P],
                "orc_classify": [P, U64, D, P, P, P, P],
                "orc_vose": [P, U64, P, P, P, P, P],
                "orc_prefix": [P, P, U64, P],
                "orc_split_binary": [P, U64, P, U64, D, P, U64, P, P, P],
                "orc_split_pary": [P, U64, P, U64, D, P, U64, U32, P, P, P],
                "orc_pary_search": [P, U64, P, U64, U32, P],
                "orc_psa": [P, U64, U64, P, P, P, P, P, P, P, U32],
                "orc_psa_prec": [P, U64, U64, ctypes.c_int, P, P],
                "orc_psa_plus": [P, U64, U64, U64, U64, P, P, P],
                "orc_mass": [P, P, U64, P],
                "orc_sample_naive": [P, P, U64, U64, U64, U64, U32, U32, P],
                "orc_sample_sectioned": [P, P, U64, U64, P, U64, U32, P],
            }
            for name, argtypes in sigs.items():
                fn = getattr(lib, name)
                fn.argtypes = argtypes
                fn.restype = ctypes.c_int
            lib.orc_philox4x32_10.argtypes = [P, P, P]
            lib.orc_philox4x32_10.restype = None
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _check(rc: int, what: str):
    if rc != OK:
        raise OracleError(rc, what)


def _f32(w) -> np.ndarray:
    return np.ascontiguousarray(w, dtype=np.float32)


def exact_sum(w) -> float:
    """W = sum w_i computed exactly, rounded once to FP64 (ties to even)."""
    w = _f32(w)
    out = np.zeros(1, np.float64)
    _check(_load().orc_exact_sum(_ptr(w), w.size, _ptr(out)), "exact_sum")
    return float(out[0])


def classify(w, avg: float):
    """Light iff (double)w_i <= avg; returns (l, h) index arrays in index order."""
    w = _f32(w)
    l = np.zeros(max(w.size, 1), np.uint32)
    h = np.zeros(max(w.size, 1), np.uint32)
    nl = np.zeros(1, np.uint64)
    nh = np.zeros(1, np.uint64)
    _check(_load().orc_classify(_ptr(w), w.size, avg, _ptr(l), _ptr(h),
                                _ptr(nl), _ptr(nh)), "classify")
    return l[: int(nl[0])].copy(), h[: int(nh[0])].copy()


def vose(w):
    """Vose's construction; returns dict(prob f64, alias u32, nl, nh, W)."""
    w = _f32(w)
    n = w.size
    prob = np.zeros(max(n, 1), np.float64)
    alias = np.zeros(max(n, 1), np.uint32)
    nl = np.zeros(1, np.uint64)
    nh = np.zeros(1, np.uint64)
    W = np.zeros(1, np.float64)
    _check(_load().orc_vose(_ptr(w), n, _ptr(prob), _ptr(alias), _ptr(nl),
                            _ptr(nh), _ptr(W)), "vose")
    return dict(prob=prob[:n], alias=alias[:n], nl=int(nl[0]), nh=int(nh[0]),
                W=float(W[0]))


def prefix(w, lst) -> np.ndarray:
    """sigma[a] = sum of w[lst[b]] for b < a, FP64, length len(lst)+1."""
    w = _f32(w)
    lst = np.ascontiguousarray(lst, dtype=np.uint32)
    sigma = np.zeros(lst.size + 1, np.float64)
    _check(_load().orc_prefix(_ptr(w), _ptr(lst), lst.size, _ptr(sigma)),
           "prefix")
    return sigma


def split_binary(sl, sh, avg: float, ks):
    """PSA splits (binary search); returns (i, j, spill) arrays."""
    sl = np.ascontiguousarray(sl, np.float64)
    sh = np.ascontiguousarray(sh, np.float64)
    ks = np.ascontiguousarray(ks, np.uint64)
    i = np.zeros(ks.size, np.uint64)
    j = np.zeros(ks.size, np.uint64)
    sp = np.zeros(ks.size, np.float64)
    _check(_load().orc_split_binary(_ptr(sl), sl.size - 1, _ptr(sh), sh.size - 1,
                                    avg, _ptr(ks), ks.size, _ptr(i), _ptr(j),
                                    _ptr(sp)), "split_binary")
    return i, j, sp


def split_pary(sl, sh, avg: float, ks, p: int):
    """PSA splits (partial p-ary search, groups of p splits)."""
    sl = np.ascontiguousarray(sl, np.float64)
    sh = np.ascontiguousarray(sh, np.float64)
    ks = np.ascontiguousarray(ks, np.uint64)
    i = np.zeros(ks.size, np.uint64)
    j = np.zeros(ks.size, np.uint64)
    sp = np.zeros(ks.size, np.float64)
    _check(_load().orc_split_pary(_ptr(sl), sl.size - 1, _ptr(sh), sh.size - 1,
                                  avg, _ptr(ks), ks.size, p, _ptr(i), _ptr(j),
                                  _ptr(sp)), "split_pary")
    return i, j, sp


def pary_search(lst, keys, p: int) -> np.ndarray:
    """Algorithm 1: upper-bound positions of sorted keys in a sorted list."""
    lst = np.ascontiguousarray(lst, np.float64)
    keys = np.ascontiguousarray(keys, np.float64)
    out = np.zeros(keys.size, np.uint64)
    _check(_load().orc_pary_search(_ptr(lst), lst.size, _ptr(keys), keys.size,
                                   p, _ptr(out)), "pary_search")
    return out


def psa(w, section: int, pary_p: int = 0):
    """PSA construction with sections of `section` buckets.

    Returns dict(prob f64, alias u32, nl, nh, split_i, split_j, spill)."""
    w = _f32(w)
    n = w.size
    nsec = (n + section - 1) // section if n else 0
    prob = np.zeros(max(n, 1), np.float64)
    alias = np.zeros(max(n, 1), np.uint32)
    nl = np.zeros(1, np.uint64)
    nh = np.zeros(1, np.uint64)
    si = np.zeros(nsec + 1, np.uint64)
    sj = np.zeros(nsec + 1, np.uint64)
    sp = np.zeros(nsec + 1, np.float64)
    _check(_load().orc_psa(_ptr(w), n, section, _ptr(prob), _ptr(alias),
                           _ptr(nl), _ptr(nh), _ptr(si), _ptr(sj), _ptr(sp),
                           pary_p), "psa")
    return dict(prob=prob[:n], alias=alias[:n], nl=int(nl[0]), nh=int(nh[0]),
                split_i=si, split_j=sj, spill=sp)


PREC_FP64, PREC_FP32_PAIR, PREC_FP32 = 0, 1, 2


def psa_prec(w, section: int, prec: int):
    """PSA (binary split search) with the prefix sums, split comparisons and
    sweep residual rounded to FP64 (prec 0), a pair of FP32 values (1, what
    compensated FP32 keeps) or plain FP32 (2).  Returns (prob f64, alias)."""
    w = _f32(w)
    n = w.size
    prob = np.zeros(max(n, 1), np.float64)
    alias = np.zeros(max(n, 1), np.uint32)
    _check(_load().orc_psa_prec(_ptr(w), n, section, prec, _ptr(prob),
                                _ptr(alias)), "psa_prec")
    return prob[:n], alias[:n]


def psa_plus(w, section: int, tile: int, min_items: int):
    """PSA+ (Sec. 4 "PSA+"): greedy packing inside each tile of `tile` items
    that holds at least `min_items` lights and heavies, then PSA (binary
    split search, sections of `section` buckets) on the unfinished items.
    Returns (prob f64, alias u32, number of items the greedy step closed)."""
    w = _f32(w)
    n = w.size
    prob = np.zeros(max(n, 1), np.float64)
    alias = np.zeros(max(n, 1), np.uint32)
    greedy = np.zeros(1, np.uint64)
    _check(_load().orc_psa_plus(_ptr(w), n, section, tile, min_items, _ptr(prob),
                                _ptr(alias), _ptr(greedy)), "psa_plus")
    return prob[:n], alias[:n], int(greedy[0])


def mass(prob, alias) -> np.ndarray:
    """mass[i] = prob[i] + sum over rows b aliasing i of (1 - prob[b])."""
    prob = np.ascontiguousarray(prob, np.float64)
    alias = np.ascontiguousarray(alias, np.uint32)
    out = np.zeros(max(prob.size, 1), np.float64)
    _check(_load().orc_mass(_ptr(prob), _ptr(alias), prob.size, _ptr(out)),
           "mass")
    return out[: prob.size]


def philox(ctr, key) -> np.ndarray:
    """One Philox-4x32-10 block for a 4-word counter and a 2-word key."""
    c = np.ascontiguousarray(ctr, np.uint32)
    k = np.ascontiguousarray(key, np.uint32)
    out = np.zeros(4, np.uint32)
    _load().orc_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def sample_naive(prob32, alias, first: int, count: int, seed: int,
                 stream_lo: int = 0, stream_hi: int = 0) -> np.ndarray:
    """Samples first..first+count-1 of Walker sampling from an FP32 table."""
    prob32 = np.ascontiguousarray(prob32, np.float32)
    alias = np.ascontiguousarray(alias, np.uint32)
    out = np.zeros(max(count, 1), np.uint32)
    _check(_load().orc_sample_naive(_ptr(prob32), _ptr(alias), prob32.size,
                                    first, count, seed, stream_lo, stream_hi,
                                    _ptr(out)), "sample_naive")
    return out[:count]


def sample_sectioned(prob32, alias, counts, seed: int, tag: int) -> np.ndarray:
    """Sectioned sampling given per-section sample counts (Sec. 5)."""
    prob32 = np.ascontiguousarray(prob32, np.float32)
    alias = np.ascontiguousarray(alias, np.uint32)
    counts = np.ascontiguousarray(counts, np.uint64)
    total = int(counts.sum())
    out = np.zeros(max(total, 1), np.uint32)
    _check(_load().orc_sample_sectioned(_ptr(prob32), _ptr(alias), prob32.size,
                                        counts.size, _ptr(counts), seed, tag,
                                        _ptr(out)), "sample_sectioned")
    return out[:total]


def expected_mass(w, W: float) -> np.ndarray:
    """N * w_i / W in FP64: the mass an exact table gives item i (Sec. 2.2)."""
    w = np.asarray(w, np.float64)
    return w * (w.size / W)


def mass_error(prob, alias, w, W: float) -> float:
    """max_i |mass_i - N w_i/W| / max(1, N w_i/W)."""
    m = mass(prob, alias)
    e = expected_mass(w, W)
    return float(np.max(np.abs(m - e) / np.maximum(1.0, e))) if m.size else 0.0
