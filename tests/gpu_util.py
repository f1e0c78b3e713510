"""Helpers shared by the GPU tests: run the CUDA path through the C ABI and
read back its outputs and intermediates."""
from __future__ import annotations

from fractions import Fraction

import numpy as np
import torch

import paper_2106_12270_gb300 as wrs


class Built:
    """Result of one GPU build: table rows, summary and workspace views."""

    def __init__(self, w_np, cfg=None, w_tensor=None, steps=False):
        self.w = np.ascontiguousarray(w_np, np.float32)
        self.n = self.w.size
        self.cfg = cfg if cfg is not None else wrs.config()
        w_dev = w_tensor if w_tensor is not None else torch.from_numpy(self.w).cuda()
        self.builder = wrs.Builder(self.n, self.cfg)
        if steps:
            rows = torch.empty(self.n, dtype=torch.int64, device="cuda")
            ws = self.builder.ws
            wrs.step_total(w_dev, ws, self.cfg)
            wrs.step_partition(w_dev, ws, self.cfg)
            wrs.step_split(self.n, ws, self.cfg)
            wrs.step_pack(self.n, rows, ws, self.cfg)
            wrs.step_info(self.n, ws, self.builder.info, self.cfg)
            self.rows_t = rows
        else:
            self.rows_t = self.builder.build(w_dev)
        torch.cuda.synchronize()
        self.info = wrs.parse_info(self.builder.info)
        self.layout = wrs.build_layout(self.n, self.cfg)
        if self.info["status"] == wrs.OK:
            self.prob, self.alias = wrs.rows_to_numpy(self.rows_t)

    # workspace views ------------------------------------------------------
    def _ws(self, off, nbytes):
        return self.builder.ws[off: off + nbytes].cpu().numpy()

    def lists(self):
        """(light items, light weights, heavy items, heavy weights) in list order."""
        raw = self._ws(self.layout["lh"], 8 * self.n).view(np.uint32).reshape(-1, 2)
        nl, nh = self.info["nl"], self.info["nh"]
        li = raw[:nl, 0].copy()
        lw = raw[:nl, 1].copy().view(np.float32)
        hraw = raw[self.n - nh:][::-1]
        return li, lw, hraw[:, 0].copy(), hraw[:, 1].copy().view(np.float32)

    def seg_pre(self, nseg):
        raw = self._ws(self.layout["seg_pre"], 48 * (nseg + 1)).view(np.uint32).reshape(-1, 12)
        out = []
        for r in raw:
            sl = sum(int(r[k]) << (32 * k) for k in range(4))
            sh = sum(int(r[4 + k]) << (32 * k) for k in range(4))
            out.append((sl, sh, int(r[8]) | int(r[9]) << 32))
        return out

    def checkpoints(self, which: str):
        """Absolute q prefix sums sigma(32c) of the light ("ckl") or heavy
        ("ckh") list, c = 0..floor(count/32)."""
        cnt = (self.info["nl"] if which == "ckl" else self.info["nh"]) // 32 + 1
        raw = self._ws(self.layout[which], 16 * cnt).view(np.uint32).reshape(-1, 4)
        segs = raw[:, 0].astype(np.int64)
        pre = self.seg_pre(int(segs.max()) if cnt else 0)
        col = 0 if which == "ckl" else 1
        return [pre[int(r[0])][col] + (int(r[2]) | int(r[3]) << 32) for r in raw]

    def splits(self):
        s = self.layout["sections"]
        raw = self._ws(self.layout["splits"], 48 * (s + 1)).view(np.uint32).reshape(-1, 12)
        i = raw[:, 0].astype(np.int64)
        j = raw[:, 1].astype(np.int64)
        D = [int(r[4]) | int(r[5]) << 32 | int(r[6]) << 64 | int(r[7]) << 96 for r in raw]
        E = [int(r[8]) | int(r[9]) << 32 | int(r[10]) << 64 | int(r[11]) << 96 for r in raw]
        return i, j, D, E


def exact_prefix(w, lst, stride):
    """Exact rational prefix sums sum_{a<i} w[lst[a]] at i = 0, stride, 2*stride..."""
    out = []
    acc = Fraction(0)
    for a, idx in enumerate(lst):
        if a % stride == 0:
            out.append(acc)
        acc += Fraction(float(w[idx]))
    if len(lst) % stride == 0:
        out.append(acc)
    return out


def gpu_sample(rows_t, n, first, count, seed, stream_lo=0, stream_hi=0, offset=0):
    """Naive samples through the C ABI; `offset` shifts the output pointer by
    whole elements to exercise unaligned outputs."""
    buf = torch.empty(count + offset + 1, dtype=torch.int32, device="cuda")
    out = buf[offset: offset + count]
    wrs.sample_rows(rows_t, n, first, count, seed, out, stream_lo, stream_hi)
    torch.cuda.synchronize()
    return out.cpu().numpy().view(np.uint32)


def fixed_q_exact(w, S):
    """q_i = floor(w_i 2^S + 1/2) for FP32 weights, exact: w 2^S is exact in
    FP64 (a 24-bit significand scaled by a power of two), the half is added
    exactly below 2^52, and from 2^52 on w 2^S is already an integer."""
    x = np.ldexp(np.asarray(w, np.float32).astype(np.float64), S)
    return np.where(x < 2.0**52, np.floor(x + 0.5), x).astype(np.uint64)


def alias_differences_at_ties(w, info, alias, orc_alias):
    """Rows whose alias differs from the oracle's PSA table, each checked to
    sit at a near-tie of the sweep's decision (Sec. 2.2: heavy h[y] closes
    before light l[x] iff its remaining weight fits in one bucket, i.e. the
    excess prefix E'(y+1) does not exceed the deficit prefix D'(x)).

    For a light row l[x] the two tables name different heavies only if some
    heavy y between them has E'(y+1) - D'(x) within the oracle's own FP64
    rounding of the two prefix sums (x + y + 2 terms, bounded by
    gamma_k * sum with gamma_k = k 2^-53 / (1 - k 2^-53)) plus the GPU's key
    resolution (2^-46 of a bucket).  The gaps are exact: D' and E' are formed
    from the fixed point q = round(w 2^S) with the build's S and Q.  Returns
    (number of differing rows, list of rows that are NOT near-ties)."""
    w = np.asarray(w, np.float32)
    n = w.size
    diff = np.flatnonzero(np.asarray(alias) != np.asarray(orc_alias))
    if diff.size == 0:
        return 0, []
    import oracle
    W = oracle.exact_sum(w)
    l, h = oracle.classify(w, W / n)
    S, Q = info["scale"], info["Q"]
    Qn = Q // n
    q = fixed_q_exact(w, S)
    ql = np.minimum(q[l], np.uint64(Qn))
    qh = np.maximum(q[h], np.uint64(Qn + 1))
    sl = np.concatenate([[0], np.cumsum(ql, dtype=np.uint64)])
    sh = np.concatenate([[0], np.cumsum(qh, dtype=np.uint64)])
    light = np.zeros(n, bool)
    light[l] = True
    eps = 2.0**-53
    bad = []
    for i in diff:
        if not light[i]:
            bad.append(int(i))   # a heavy closes with the next heavy in both tables
            continue
        x = int(np.searchsorted(l, i))
        ya = int(np.searchsorted(h, alias[i]))
        yb = int(np.searchsorted(h, orc_alias[i]))
        D = x * Q - n * int(sl[x])
        tie = False
        for y in range(min(ya, yb), max(ya, yb)):
            E = n * int(sh[y + 1]) - (y + 1) * Q
            k = x + y + 2
            gamma = k * eps / (1.0 - k * eps)
            # the two FP64 prefix sums in buckets: N sigma / Q
            bound = gamma * n * (float(sl[x]) + float(sh[y + 1])) / Q + 2.0**-46
            tie = tie or abs(E - D) / Q <= bound
        if not tie:
            bad.append(int(i))
    return int(diff.size), bad
