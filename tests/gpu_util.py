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
