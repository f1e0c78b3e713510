"""Alias-table construction and sampling on GB300 (sm_103a).

Thin Python binding of the C ABI declared in ``include/wrs.h``: every
function here only marshals arguments (torch tensors for device memory,
torch streams) and calls ``libwrs.so``; every step of the computation runs
in the library's CUDA kernels.  There is no CPU fallback: if the library is
missing or no GPU is present, calls raise.

Method: "Weighted Random Sampling on GPUs" (Lehmann, Huebschle-Schneider,
Sanders, arXiv 2106.12270) -- PSA construction (Sec. 2.2, Sec. 4) and
Walker / sectioned sampling (Sec. 2.2, Sec. 5).
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import _build

__all__ = [
    "WrsError", "lib", "config", "build_workspace_bytes", "build_layout", "build_rows",
    "step_total", "step_partition", "step_split", "step_pack", "step_info", "sample_rows",
    "parse_info", "INFO_BYTES", "BatchTuning", "ROW_BYTES", "Builder", "rows_to_numpy",
    "build_plus_workspace_bytes", "build_rows_plus",
]

OK, EINVAL, EZEROSUM, ENONFINITE, ENOMEM, ETIMEOUT, ECUDA, EBUSY, ENOTFOUND = range(9)
SPLIT_PARY, SPLIT_BINARY = 0, 1
SAMPLE_NAIVE, SAMPLE_CACHED, SAMPLE_LIMITED, SAMPLE_SMEM, SAMPLE_AUTO = 0, 1, 2, 3, 4
TAG_NAIVE, TAG_SECTION, TAG_COUNTS, TAG_BATCH, TAG_DIAG = 0, 1, 2, 3, 4
ROW_BYTES = 8

_lock = threading.Lock()
_lib = None


class WrsError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        msg = lib().wrs_strerror(status).decode() if _lib is not None else str(status)
        super().__init__(f"{what}: wrs status {status} ({msg})")
        self.status = status


class Config(ctypes.Structure):
    _fields_ = [("section_size", ctypes.c_uint32), ("split_method", ctypes.c_uint32),
                ("reserved", ctypes.c_uint32 * 6)]


class Layout(ctypes.Structure):
    _fields_ = [("lh", ctypes.c_uint64), ("ckl", ctypes.c_uint64), ("ckh", ctypes.c_uint64),
                ("seg_pre", ctypes.c_uint64), ("splits", ctypes.c_uint64),
                ("sections", ctypes.c_uint64), ("total_bytes", ctypes.c_uint64)]


class BatchTuning(ctypes.Structure):
    """Tiling of the batched build (wrs_batch_tuning)."""
    _fields_ = [("threads", ctypes.c_uint32), ("chunk", ctypes.c_uint32),
                ("ctas_per_sm", ctypes.c_uint32), ("ms", ctypes.c_float),
                ("reserved", ctypes.c_uint32 * 4)]

    def as_dict(self) -> dict:
        return {"threads": self.threads, "chunk": self.chunk, "ctas_per_sm": self.ctas_per_sm,
                "ms": self.ms}


class ServerStats(ctypes.Structure):
    _fields_ = [("completed", ctypes.c_uint64), ("builds", ctypes.c_uint64),
                ("samples", ctypes.c_uint64), ("releases", ctypes.c_uint64),
                ("errors", ctypes.c_uint64), ("items_built", ctypes.c_uint64),
                ("samples_drawn", ctypes.c_uint64), ("steps", ctypes.c_uint64),
                ("mean_step_requests", ctypes.c_double), ("resident_bytes", ctypes.c_uint64),
                ("peak_bytes", ctypes.c_uint64), ("p50_ms", ctypes.c_double),
                ("p99_ms", ctypes.c_double), ("mean_ms", ctypes.c_double),
                ("wall_s", ctypes.c_double)]


INFO_DTYPE = np.dtype([("status", "<i4"), ("scale", "<i4"), ("W", "<f8"), ("avg", "<f8"),
                       ("nl", "<u8"), ("nh", "<u8"), ("Q", "<u4", (4,)),
                       ("light_max", "<f4"), ("sections", "<u4"), ("reserved", "<u8", (4,))])
INFO_BYTES = INFO_DTYPE.itemsize


def lib():
    """Load libwrs.so (built by __graft_entry__.build()); raise if it is missing."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(_build.LIB):
                raise RuntimeError(f"{_build.LIB} is missing: build the CUDA library first "
                                   "(python -c 'import __graft_entry__ as g; g.build()')")
            L = ctypes.CDLL(_build.LIB)
            P, U64, U32, I = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int
            CP = ctypes.POINTER(Config)
            sigs = {
                "wrs_build_workspace_bytes": (I, [U64, CP, ctypes.POINTER(U64)]),
                "wrs_build_layout": (I, [U64, CP, ctypes.POINTER(Layout)]),
                "wrs_build_rows": (I, [P, U64, P, P, U64, CP, P, P]),
                "wrs_build_rows_noalloc": (I, [P, U64, P, CP, P, P]),
                "wrs_build_host_workspace_bytes": (I, [U64, CP, ctypes.POINTER(U64)]),
                "wrs_build_rows_host": (I, [P, U64, P, P, U64, CP, P, P]),
                "wrs_step_total": (I, [P, U64, P, U64, CP, P]),
                "wrs_step_partition": (I, [P, U64, P, U64, CP, P]),
                "wrs_step_split": (I, [U64, P, U64, CP, P]),
                "wrs_step_pack": (I, [U64, P, P, U64, CP, P]),
                "wrs_step_info": (I, [U64, P, U64, CP, P, P]),
                "wrs_sample_rows": (I, [P, U64, U64, U64, U64, U32, U32, P, P]),
                "wrs_diag_random_gather": (I, [P, U64, U64, U64, I, U32, U32, P, P]),
                "wrs_diag_build_each": (I, [P, P, U32, P, P, U64, CP, P, P]),
                "wrs_set_config": (I, [CP]),
                "wrs_get_config": (I, [CP]),
                "wrs_build": (I, [P, U64, I, P, ctypes.POINTER(P)]),
                "wrs_sample": (I, [P, U64, U64, P, I, P]),
                "wrs_table_info": (I, [P, ctypes.POINTER(U64), ctypes.POINTER(ctypes.c_double),
                                       ctypes.POINTER(U64), ctypes.POINTER(U64)]),
                "wrs_table_rows": (I, [P, ctypes.POINTER(P)]),
                "wrs_table_export": (I, [P, P, I]),
                "wrs_table_import": (I, [P, U64, I, ctypes.c_double, ctypes.POINTER(P)]),
                "wrs_table_destroy": (I, [P]),
                "wrs_build_batched": (I, [P, P, U32, P, ctypes.POINTER(P)]),
                "wrs_batch_status": (I, [P, P]),
                "wrs_batch_summaries": (I, [P, P]),
                "wrs_batch_rows": (I, [P, ctypes.POINTER(P), ctypes.POINTER(P),
                                       ctypes.POINTER(U32)]),
                "wrs_sample_batched": (I, [P, P, U64, P, P]),
                "wrs_batch_export": (I, [P, P, I]),
                "wrs_batch_destroy": (I, [P]),
                "wrs_diag_philox": (I, [U64, U64, P, P]),
                "wrs_diag_prec_workspace_bytes": (I, [U64, CP, ctypes.POINTER(U64)]),
                "wrs_diag_prec_split_pack": (I, [U64, P, P, U64, P, U64, CP, U32, P]),
                "wrs_diag_pack_variant": (I, [P, U64, P, P, U64, P, U32, P]),
                "wrs_build_plus_workspace_bytes": (I, [U64, P, ctypes.POINTER(U64)]),
                "wrs_build_rows_plus": (I, [P, U64, P, P, U64, P, U32, P, ctypes.POINTER(U64), P]),
                "wrs_sample_sections": (I, [U64, U32, ctypes.POINTER(U64)]),
                "wrs_sample_auto_choice": (I, [U64, U64, ctypes.POINTER(U32),
                                               ctypes.POINTER(U32)]),
                "wrs_sample_auto_workspace_bytes": (I, [U64, U64, ctypes.POINTER(U64)]),
                "wrs_sample_auto": (I, [P, U64, U64, U64, P, P, U64, ctypes.POINTER(U32), P]),
                "wrs_build_batched_workspace_bytes": (I, [U64, U32, ctypes.POINTER(U64)]),
                "wrs_batch_order": (I, [P, U32, P]),
                "wrs_build_batched_rows": (I, [P, P, U32, P, P, P, U64, P, P]),
                "wrs_build_batched_rows_tuned": (I, [P, P, U32, P, P, P, U64, P,
                                                     ctypes.POINTER(BatchTuning), P]),
                "wrs_batch_tuning_default": (I, [ctypes.POINTER(BatchTuning)]),
                "wrs_batch_autotune": (I, [P, P, U32, P, P, P, U64, P, P, I,
                                           ctypes.POINTER(BatchTuning),
                                           ctypes.POINTER(BatchTuning), ctypes.POINTER(U32)]),
                "wrs_sample_batched_rows": (I, [P, P, U32, P, U64, P, P]),
                "wrs_server_create": (I, [U64, U32, ctypes.POINTER(P)]),
                "wrs_server_submit_build": (I, [P, P, U64, I, ctypes.POINTER(U64)]),
                "wrs_server_submit_sample": (I, [P, U64, U64, U64, U32, P, I,
                                                 ctypes.POINTER(U64)]),
                "wrs_server_submit_release": (I, [P, U64, ctypes.POINTER(U64)]),
                "wrs_server_poll": (I, [P, U64, ctypes.POINTER(I), ctypes.POINTER(I)]),
                "wrs_server_wait": (I, [P, U64, ctypes.POINTER(I)]),
                "wrs_server_table": (I, [P, U64, ctypes.POINTER(P), ctypes.POINTER(U64),
                                         ctypes.POINTER(ctypes.c_double)]),
                "wrs_server_stats": (I, [P, ctypes.POINTER(ServerStats)]),
                "wrs_server_export": (I, [P, U64, P, I]),
                "wrs_server_destroy": (I, [P]),
                "wrs_sample_sectioned_rows": (I, [P, U64, U64, U64, U32, U32, P, P, P, P]),
                "wrs_strerror": (ctypes.c_char_p, [I]),
                "wrs_last_cuda_error": (I, []),
                "wrs_abi_version": (I, []),
                "wrs_config_default": (None, [CP]),
            }
            for name, (res, args) in sigs.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def config(section_size: int = 1024, split_method: int = SPLIT_PARY) -> Config:
    c = Config()
    lib().wrs_config_default(ctypes.byref(c))
    c.section_size = section_size
    c.split_method = split_method
    return c


def _cfg(cfg):
    return ctypes.byref(cfg) if cfg is not None else None


def _stream(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _check(rc: int, what: str):
    if rc != OK:
        raise WrsError(rc, what)


def build_workspace_bytes(n: int, cfg: Config | None = None) -> int:
    out = ctypes.c_uint64()
    _check(lib().wrs_build_workspace_bytes(n, _cfg(cfg), ctypes.byref(out)),
           "wrs_build_workspace_bytes")
    return out.value


def build_layout(n: int, cfg: Config | None = None) -> dict:
    out = Layout()
    _check(lib().wrs_build_layout(n, _cfg(cfg), ctypes.byref(out)), "wrs_build_layout")
    return {f: getattr(out, f) for f, _ in Layout._fields_}


def build_rows(w, rows, ws, info, cfg: Config | None = None, stream=None):
    """Enqueue a full build (Sec. 2.2, Sec. 4): w (float32 [n], device) ->
    rows (int64 [n], device, {prob, alias} per row)."""
    n = w.numel()
    if rows.numel() < n or rows.element_size() != 8:
        raise ValueError("build_rows: rows must hold n 8-byte rows")
    _check(lib().wrs_build_rows(_ptr(w), n, _ptr(rows), _ptr(ws), ws.numel() * ws.element_size(),
                                _cfg(cfg), _ptr(info), _stream(stream)), "wrs_build_rows")


def _same_device(what: str, dev, *tensors):
    for t in tensors:
        if t is not None and t.device != dev:
            raise ValueError(f"{what}: every tensor must be on {dev}, got {t.device}")


def build_rows_noalloc(w, rows, info, cfg: Config | None = None, stream=None):
    """Enqueue a full build that allocates nothing (workspace inside the
    library; n <= 3.5 million; calls on one device must not overlap).
    w: float32 [n], rows: int64 [n], info: uint8 [INFO_BYTES], all on one
    CUDA device; the call runs with that device current."""
    import torch
    n = w.numel()
    if not w.is_cuda:
        raise ValueError("build_rows_noalloc: weights must be on a CUDA device")
    _same_device("build_rows_noalloc", w.device, rows, info)
    if w.dtype != torch.float32 or rows.dtype != torch.int64 or rows.numel() != n:
        raise ValueError("build_rows_noalloc: w must be float32 [n] and rows int64 [n]")
    if info.numel() * info.element_size() < INFO_BYTES:
        raise ValueError("build_rows_noalloc: info holds fewer than INFO_BYTES bytes")
    if stream is not None and stream.device != w.device:
        raise ValueError("build_rows_noalloc: the stream is on another device")
    with torch.cuda.device(w.device):
        _check(lib().wrs_build_rows_noalloc(_ptr(w), n, _ptr(rows), _cfg(cfg), _ptr(info),
                                            _stream(stream)), "wrs_build_rows_noalloc")


def build_host_workspace_bytes(n: int, cfg: Config | None = None) -> int:
    out = ctypes.c_uint64()
    _check(lib().wrs_build_host_workspace_bytes(n, _cfg(cfg), ctypes.byref(out)),
           "wrs_build_host_workspace_bytes")
    return out.value


def build_rows_host(w_host, rows_host, ws, info_host, cfg: Config | None = None, stream=None):
    """Enqueue a build from host memory (wrs_build_rows_host): w_host (float32
    [n], host, pinned for an asynchronous call) -> rows_host (int64 [n], host);
    info_host: uint8 [INFO_BYTES] host tensor for the summary."""
    n = w_host.numel()
    _check(lib().wrs_build_rows_host(_ptr(w_host), n, _ptr(rows_host), _ptr(ws),
                                     ws.numel() * ws.element_size(), _cfg(cfg), _ptr(info_host),
                                     _stream(stream)), "wrs_build_rows_host")


def step_total(w, ws, cfg=None, stream=None):
    _check(lib().wrs_step_total(_ptr(w), w.numel(), _ptr(ws), ws.numel() * ws.element_size(),
                                _cfg(cfg), _stream(stream)), "wrs_step_total")


def step_partition(w, ws, cfg=None, stream=None):
    _check(lib().wrs_step_partition(_ptr(w), w.numel(), _ptr(ws), ws.numel() * ws.element_size(),
                                    _cfg(cfg), _stream(stream)), "wrs_step_partition")


def step_split(n, ws, cfg=None, stream=None):
    _check(lib().wrs_step_split(n, _ptr(ws), ws.numel() * ws.element_size(), _cfg(cfg),
                                _stream(stream)), "wrs_step_split")


def step_pack(n, rows, ws, cfg=None, stream=None):
    _check(lib().wrs_step_pack(n, _ptr(rows), _ptr(ws), ws.numel() * ws.element_size(),
                               _cfg(cfg), _stream(stream)), "wrs_step_pack")


def step_info(n, ws, info, cfg=None, stream=None):
    _check(lib().wrs_step_info(n, _ptr(ws), ws.numel() * ws.element_size(), _cfg(cfg),
                               _ptr(info), _stream(stream)), "wrs_step_info")


def sample_rows(rows, n: int, first: int, count: int, seed: int, out,
                stream_lo: int = 0, stream_hi: int = TAG_NAIVE, stream=None):
    """Enqueue naive Walker sampling (Sec. 2.2, Sec. 5): samples
    first..first+count-1 of stream (seed, stream_lo, stream_hi) into out
    (int32/uint32 [count], device)."""
    _check(lib().wrs_sample_rows(_ptr(rows), n, first, count, seed & (2**64 - 1), stream_lo,
                                 stream_hi, _ptr(out), _stream(stream)), "wrs_sample_rows")


def sample_sections(n: int, section_rows: int) -> int:
    out = ctypes.c_uint64()
    _check(lib().wrs_sample_sections(n, section_rows, ctypes.byref(out)), "wrs_sample_sections")
    return out.value


def sample_sectioned_rows(rows, n: int, count: int, seed: int, mode: int, section_rows: int,
                          counts, offsets, out, stream=None):
    """Enqueue sectioned sampling (Sec. 5): per-section counts/offsets
    (int64 [nsec], device) and samples grouped by section in out."""
    _check(lib().wrs_sample_sectioned_rows(_ptr(rows), n, count, seed & (2**64 - 1), mode,
                                           section_rows, _ptr(counts), _ptr(offsets), _ptr(out),
                                           _stream(stream)), "wrs_sample_sectioned_rows")


MODE_NAMES = {0: "naive", 1: "cached", 2: "limited", 3: "smem"}


def sample_auto_plan(n: int, count: int):
    """(mode code, rows per section) that wrs_sample_auto uses for n rows and
    count draws (rows per section is 0 for naive sampling)."""
    mode, rows = ctypes.c_uint32(), ctypes.c_uint32()
    _check(lib().wrs_sample_auto_choice(n, count, ctypes.byref(mode), ctypes.byref(rows)),
           "wrs_sample_auto_choice")
    return mode.value, rows.value


def sample_auto_choice(n: int, count: int) -> str:
    """The sampling mode wrs_sample_auto picks for n rows and count draws."""
    return MODE_NAMES[sample_auto_plan(n, count)[0]]


def sample_auto(rows, n: int, count: int, seed: int, out, stream=None) -> str:
    """Draw count samples with the automatically chosen mode (wrs_sample_auto);
    returns the mode's name.  The workspace is a torch tensor on the device."""
    import torch
    nb = ctypes.c_uint64()
    _check(lib().wrs_sample_auto_workspace_bytes(n, count, ctypes.byref(nb)),
           "wrs_sample_auto_workspace_bytes")
    ws = torch.empty(max(nb.value, 256), dtype=torch.uint8, device=rows.device)
    used = ctypes.c_uint32()
    _check(lib().wrs_sample_auto(_ptr(rows), n, count, seed & (2**64 - 1), _ptr(out), _ptr(ws),
                                 ws.numel(), ctypes.byref(used), _stream(stream)),
           "wrs_sample_auto")
    return MODE_NAMES[used.value]


SUMMARY_DTYPE = np.dtype([("status", "<i4"), ("n", "<u4"), ("W", "<f8"), ("nl", "<u8"),
                          ("nh", "<u8")])


def batch_order(off_host) -> np.ndarray:
    """Host plan: table ids largest first (wrs_batch_order)."""
    off = np.ascontiguousarray(off_host, np.uint64)
    ntab = off.size - 1
    order = np.zeros(max(ntab, 1), np.uint32)
    _check(lib().wrs_batch_order(off.ctypes.data_as(ctypes.c_void_p), ntab,
                                 order.ctypes.data_as(ctypes.c_void_p)), "wrs_batch_order")
    return order[:ntab]


class BatchBuilder:
    """Workspace and buffers for building a batch of tables in one launch
    (wrs_build_batched_rows); all arguments are torch tensors on the GPU."""

    def __init__(self, total: int, ntab: int, device="cuda"):
        import torch
        out = ctypes.c_uint64()
        _check(lib().wrs_build_batched_workspace_bytes(total, ntab, ctypes.byref(out)),
               "wrs_build_batched_workspace_bytes")
        self.ws = torch.empty(out.value, dtype=torch.uint8, device=device)
        self.info = torch.zeros(max(ntab, 1) * SUMMARY_DTYPE.itemsize, dtype=torch.uint8,
                                device=device)
        self.ntab = ntab
        self.tuning = None   # None: the default tiling

    def build(self, w, off, rows, order=None, stream=None):
        """Enqueue the batched build with the current tiling (self.tuning)."""
        t = ctypes.byref(self.tuning) if self.tuning is not None else None
        _check(lib().wrs_build_batched_rows_tuned(_ptr(w), _ptr(off), self.ntab, _ptr(order),
                                                  _ptr(rows), _ptr(self.ws), self.ws.numel(),
                                                  _ptr(self.info), t, _stream(stream)),
               "wrs_build_batched_rows_tuned")

    def autotune(self, w, off, rows, order=None, stream=None, force=False):
        """Time every candidate tiling on this batch (wrs_batch_autotune), keep
        the fastest for later builds; returns (best, all candidates) as dicts.
        The rows hold a valid build afterwards."""
        best = BatchTuning()
        cand = (BatchTuning * 16)()
        nall = ctypes.c_uint32(16)
        _check(lib().wrs_batch_autotune(_ptr(w), _ptr(off), self.ntab, _ptr(order), _ptr(rows),
                                        _ptr(self.ws), self.ws.numel(), _ptr(self.info),
                                        _stream(stream), int(force), ctypes.byref(best), cand,
                                        ctypes.byref(nall)), "wrs_batch_autotune")
        self.tuning = best
        return best.as_dict(), [cand[k].as_dict() for k in range(min(nall.value, 16))]

    def summaries(self) -> np.ndarray:
        raw = self.info.cpu().numpy().tobytes()
        return np.frombuffer(raw, SUMMARY_DTYPE, count=self.ntab)


def sample_batched_rows(rows, off, ntab: int, cnt_off, seed: int, out, stream=None):
    """Enqueue batched sampling (wrs_sample_batched_rows)."""
    _check(lib().wrs_sample_batched_rows(_ptr(rows), _ptr(off), ntab, _ptr(cnt_off),
                                         seed & (2**64 - 1), _ptr(out), _stream(stream)),
           "wrs_sample_batched_rows")


class Server:
    """Request loop over resident tables (wrs_server_*).  Weights and sample
    outputs are torch tensors (host or device); they must stay alive until
    the request is done, which this class ensures by holding references."""

    def __init__(self, hbm_budget: int, max_inflight: int = 2):
        h = ctypes.c_void_p()
        _check(lib().wrs_server_create(hbm_budget, max_inflight, ctypes.byref(h)),
               "wrs_server_create")
        self.h = h
        self._keep = {}

    def build(self, w) -> int:
        t = ctypes.c_uint64()
        _check(lib().wrs_server_submit_build(self.h, _ptr(w), w.numel(), int(w.is_cuda),
                                             ctypes.byref(t)), "wrs_server_submit_build")
        self._keep[t.value] = w
        return t.value

    def sample(self, table: int, count: int, seed: int, out, stream_lo: int = 0) -> int:
        t = ctypes.c_uint64()
        _check(lib().wrs_server_submit_sample(self.h, table, count, seed & (2**64 - 1), stream_lo,
                                              _ptr(out), int(out.is_cuda), ctypes.byref(t)),
               "wrs_server_submit_sample")
        self._keep[t.value] = out
        return t.value

    def release(self, table: int) -> int:
        t = ctypes.c_uint64()
        _check(lib().wrs_server_submit_release(self.h, table, ctypes.byref(t)),
               "wrs_server_submit_release")
        return t.value

    def poll(self, ticket: int):
        d, s = ctypes.c_int(), ctypes.c_int()
        _check(lib().wrs_server_poll(self.h, ticket, ctypes.byref(d), ctypes.byref(s)),
               "wrs_server_poll")
        return bool(d.value), s.value

    def wait(self, ticket: int) -> int:
        s = ctypes.c_int()
        _check(lib().wrs_server_wait(self.h, ticket, ctypes.byref(s)), "wrs_server_wait")
        self._keep.pop(ticket, None)
        return s.value

    def table(self, table: int):
        """(device pointer, n, W) of a built, resident table."""
        p, n, W = ctypes.c_void_p(), ctypes.c_uint64(), ctypes.c_double()
        _check(lib().wrs_server_table(self.h, table, ctypes.byref(p), ctypes.byref(n),
                                      ctypes.byref(W)), "wrs_server_table")
        return p.value, n.value, W.value

    def export(self, table: int, dst):
        """Copy a resident table's rows into dst (int64 [n], host or device)."""
        _check(lib().wrs_server_export(self.h, table, _ptr(dst), int(dst.is_cuda)),
               "wrs_server_export")
        return dst

    def stats(self) -> dict:
        st = ServerStats()
        _check(lib().wrs_server_stats(self.h, ctypes.byref(st)), "wrs_server_stats")
        return {f: getattr(st, f) for f, _ in ServerStats._fields_}

    def close(self):
        if self.h:
            _check(lib().wrs_server_destroy(self.h), "wrs_server_destroy")
            self.h = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def diag_random_gather(rows, nrows: int, count: int, seed: int, flavor: int, out,
                       ctas_per_sm: int = 8, loads_in_flight: int = 8, stream=None):
    """Enqueue the random-gather probe (measurement support, not the method)."""
    _check(lib().wrs_diag_random_gather(_ptr(rows), nrows, count, seed, flavor, ctas_per_sm,
                                        loads_in_flight, _ptr(out), _stream(stream)),
           "wrs_diag_random_gather")


def diag_build_each(w, off_host, rows, reps: int = 1, cfg: Config | None = None, stream=None):
    """Build every table of a batch (weights w, host offsets off_host, rows
    as for the batched build) with its own launch sequence of the
    single-table pipeline (wrs_diag_build_each), `reps` times; returns (mean
    ms per pass from CUDA events, number of tables whose status is not OK)."""
    import torch
    off = np.ascontiguousarray(off_host, np.uint64)
    ntab = off.size - 1
    sizes = off[1:] - off[:-1]
    cap = int(sizes.max()) if ntab else 1
    ws = torch.empty(build_workspace_bytes(max(cap, 1), cfg), dtype=torch.uint8, device=w.device)
    info = torch.zeros(max(ntab, 1) * INFO_BYTES, dtype=torch.uint8, device=w.device)
    st = torch.cuda.current_stream() if stream is None else stream

    def once():
        _check(lib().wrs_diag_build_each(_ptr(w), off.ctypes.data_as(ctypes.c_void_p), ntab,
                                         _ptr(rows), _ptr(ws), ws.numel(), _cfg(cfg), _ptr(info),
                                         ctypes.c_void_p(st.cuda_stream)), "wrs_diag_build_each")

    once()
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(st)
    for _ in range(reps):
        once()
    b.record(st)
    torch.cuda.synchronize()
    raw = info.cpu().numpy()[: ntab * INFO_BYTES].tobytes()
    recs = np.frombuffer(raw, INFO_DTYPE, count=ntab)
    bad = int(((recs["status"] != OK) & (sizes > 0)).sum())
    return a.elapsed_time(b) / reps, bad


def build_plus_workspace_bytes(n: int, cfg: Config | None = None) -> int:
    out = ctypes.c_uint64()
    _check(lib().wrs_build_plus_workspace_bytes(n, _cfg(cfg), ctypes.byref(out)),
           "wrs_build_plus_workspace_bytes")
    return out.value


def build_rows_plus(w, rows, ws, info, cfg: Config | None = None, min_items: int = 1,
                    stream=None) -> int:
    """PSA+ build (Sec. 4): w (float32 [n], device) -> rows (int64 [n],
    device); greedy packing in chunks with at least min_items light and heavy
    items, PSA on the rest.  Returns how many items the greedy step finished;
    synchronises the stream once."""
    n = w.numel()
    greedy = ctypes.c_uint64()
    _check(lib().wrs_build_rows_plus(_ptr(w), n, _ptr(rows), _ptr(ws),
                                     ws.numel() * ws.element_size(), _cfg(cfg), min_items,
                                     _ptr(info), ctypes.byref(greedy),
                                     _stream(stream)), "wrs_build_rows_plus")
    return greedy.value


def diag_pack_variant(w, n: int, rows, ws, cfg: Config | None = None, variant: int = 1,
                      stream=None):
    """Pack step by one of the paper's sequential pack designs (Sec. 4.2,
    Fig. 3) on a workspace after step_split; same rows as step_pack."""
    _check(lib().wrs_diag_pack_variant(_ptr(w), n, _ptr(rows),
                                       _ptr(ws), ws.numel() * ws.element_size(), _cfg(cfg),
                                       variant, _stream(stream)), "wrs_diag_pack_variant")


PREC_FP64, PREC_FF = 0, 1


def diag_prec_workspace_bytes(n: int, cfg: Config | None = None) -> int:
    out = ctypes.c_uint64()
    _check(lib().wrs_diag_prec_workspace_bytes(n, _cfg(cfg), ctypes.byref(out)),
           "wrs_diag_prec_workspace_bytes")
    return out.value


def diag_prec_split_pack(n: int, rows, ws, pws, cfg: Config | None = None,
                         prec: int = PREC_FP64, stream=None):
    """Split and pack with FP64 (prec 0) or paired-FP32 (prec 1) prefix
    arithmetic on a build's lists (ws after step_partition): the precision
    study of Sec. 2.2's prefix sums (measurement, not the library's build)."""
    _check(lib().wrs_diag_prec_split_pack(n, _ptr(rows), _ptr(ws), ws.numel() * ws.element_size(),
                                          _ptr(pws), pws.numel() * pws.element_size(), _cfg(cfg),
                                          prec, _stream(stream)), "wrs_diag_prec_split_pack")


def diag_philox(count: int, seed: int, out, stream=None):
    """Enqueue the Philox-rate probe (measurement support, not the method)."""
    _check(lib().wrs_diag_philox(count, seed, _ptr(out), _stream(stream)), "wrs_diag_philox")


def parse_info(info_tensor) -> dict:
    """Decode a device wrs_build_info (uint8 [INFO_BYTES]) after the stream synced."""
    raw = info_tensor.detach().cpu().numpy().tobytes()
    rec = np.frombuffer(raw, INFO_DTYPE, count=1)[0]
    q = [int(x) for x in rec["Q"]]
    return dict(status=int(rec["status"]), scale=int(rec["scale"]), W=float(rec["W"]),
                avg=float(rec["avg"]), nl=int(rec["nl"]), nh=int(rec["nh"]),
                Q=q[0] | q[1] << 32 | q[2] << 64 | q[3] << 96,
                light_max=float(rec["light_max"]), sections=int(rec["sections"]))


def rows_to_numpy(rows):
    """Split an int64 row tensor into (prob float32, alias uint32) numpy arrays."""
    a = rows.detach().cpu().numpy().view(np.uint32).reshape(-1, 2)
    return a[:, 0].copy().view(np.float32), a[:, 1].copy()


class Builder:
    """Owns a build workspace sized for up to `capacity` items and builds
    tables into caller-provided row tensors."""

    def __init__(self, capacity: int, cfg: Config | None = None, device="cuda"):
        import torch
        self.cfg = cfg if cfg is not None else config()
        self.capacity = capacity
        nbytes = build_workspace_bytes(capacity, self.cfg)
        self.ws = torch.empty(nbytes, dtype=torch.uint8, device=device)
        self.info = torch.zeros(INFO_BYTES, dtype=torch.uint8, device=device)

    def build(self, w, rows=None, stream=None):
        import torch
        n = w.numel()
        if n > self.capacity:
            raise ValueError("table larger than the workspace capacity")
        if rows is None:
            rows = torch.empty(n, dtype=torch.int64, device=w.device)
        build_rows(w, rows, self.ws, self.info, self.cfg, stream)
        return rows


# ---------------------------------------------------------------------------
# Table and batch objects (wrs_build / wrs_sample / wrs_table_* / wrs_batch_*)
# ---------------------------------------------------------------------------

def set_config(cfg: Config):
    """Process-wide build settings of Table.build (wrs_set_config)."""
    _check(lib().wrs_set_config(ctypes.byref(cfg)), "wrs_set_config")


def get_config() -> Config:
    c = Config()
    _check(lib().wrs_get_config(ctypes.byref(c)), "wrs_get_config")
    return c


class Table:
    """An alias table owned by the library (wrs_table).  Build it from
    weights (a torch tensor on the device or the host, or a numpy array),
    sample it, export and import its rows."""

    def __init__(self, handle):
        self.h = handle

    @classmethod
    def build(cls, w, stream=None) -> "Table":
        """wrs_build: weights (float32, 1-D) -> table; raises WrsError on a
        data error (negative, non-finite or all-zero weights)."""
        import torch
        if isinstance(w, np.ndarray):
            w = torch.from_numpy(np.ascontiguousarray(w, np.float32))
        if w.dtype != torch.float32 or w.dim() != 1 or not w.is_contiguous():
            raise ValueError("weights must be a contiguous 1-D float32 tensor")
        h = ctypes.c_void_p()
        _check(lib().wrs_build(_ptr(w), w.numel(), int(w.is_cuda), _stream(stream),
                               ctypes.byref(h)), "wrs_build")
        return cls(h)

    @classmethod
    def import_rows(cls, rows, W: float = float("nan")) -> "Table":
        """wrs_table_import: rows (int64 tensor, host or device) -> table."""
        h = ctypes.c_void_p()
        _check(lib().wrs_table_import(_ptr(rows), rows.numel(), int(rows.is_cuda), W,
                                      ctypes.byref(h)), "wrs_table_import")
        return cls(h)

    def sample(self, count: int, seed: int, out, mode: int = SAMPLE_NAIVE, stream=None):
        """wrs_sample: count draws into out (int32/uint32 tensor on the device)."""
        _check(lib().wrs_sample(self.h, count, seed & (2**64 - 1), _ptr(out), mode,
                                _stream(stream)), "wrs_sample")
        return out

    def info(self) -> dict:
        n, W, nl, nh = ctypes.c_uint64(), ctypes.c_double(), ctypes.c_uint64(), ctypes.c_uint64()
        _check(lib().wrs_table_info(self.h, ctypes.byref(n), ctypes.byref(W), ctypes.byref(nl),
                                    ctypes.byref(nh)), "wrs_table_info")
        return {"n": n.value, "W": W.value, "nl": nl.value, "nh": nh.value}

    def rows_ptr(self) -> int:
        p = ctypes.c_void_p()
        _check(lib().wrs_table_rows(self.h, ctypes.byref(p)), "wrs_table_rows")
        return p.value

    def export(self, dst=None, device=False):
        """wrs_table_export into dst (int64 [n], host or device; allocated
        on the host, or the device if device=True, when dst is None)."""
        import torch
        n = self.info()["n"]
        if dst is None:
            dst = torch.empty(n, dtype=torch.int64, device="cuda" if device else "cpu")
        _check(lib().wrs_table_export(self.h, _ptr(dst), int(dst.is_cuda)), "wrs_table_export")
        return dst

    def close(self):
        if self.h:
            _check(lib().wrs_table_destroy(self.h), "wrs_table_destroy")
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Many tables built in one launch (wrs_build_batched / wrs_batch_*)."""

    def __init__(self, handle):
        self.h = handle

    @classmethod
    def build(cls, w, off, stream=None) -> "Batch":
        """w: float32 device tensor of all tables' weights; off: int64 device
        tensor of ntab+1 offsets."""
        h = ctypes.c_void_p()
        _check(lib().wrs_build_batched(_ptr(w), _ptr(off), off.numel() - 1, _stream(stream),
                                       ctypes.byref(h)), "wrs_build_batched")
        return cls(h)

    def _rows(self):
        r, o, nt = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_uint32()
        _check(lib().wrs_batch_rows(self.h, ctypes.byref(r), ctypes.byref(o), ctypes.byref(nt)),
               "wrs_batch_rows")
        return r.value, o.value, nt.value

    @property
    def ntab(self) -> int:
        return self._rows()[2]

    def status(self) -> np.ndarray:
        st = np.zeros(max(self.ntab, 1), np.int32)
        _check(lib().wrs_batch_status(self.h, st.ctypes.data_as(ctypes.c_void_p)),
               "wrs_batch_status")
        return st[: self.ntab]

    def summaries(self) -> np.ndarray:
        out = np.zeros(max(self.ntab, 1), SUMMARY_DTYPE)
        _check(lib().wrs_batch_summaries(self.h, out.ctypes.data_as(ctypes.c_void_p)),
               "wrs_batch_summaries")
        return out[: self.ntab]

    def export(self, dst):
        """wrs_batch_export: copy all rows of the batch (table-local aliases)
        into dst (int64 [total items], host or device)."""
        _check(lib().wrs_batch_export(self.h, _ptr(dst), int(dst.is_cuda)), "wrs_batch_export")
        return dst

    def sample(self, cnt_off, seed: int, out, stream=None):
        _check(lib().wrs_sample_batched(self.h, _ptr(cnt_off), seed & (2**64 - 1), _ptr(out),
                                        _stream(stream)), "wrs_sample_batched")
        return out

    def close(self):
        if self.h:
            _check(lib().wrs_batch_destroy(self.h), "wrs_batch_destroy")
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
