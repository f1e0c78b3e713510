"""The C ABI library builds for sm_103a, loads, and exports every entry point
that include/wrs.h declares; host-side argument checks work without a GPU
(no compute call is made here)."""
from __future__ import annotations

import ctypes
import os
import re

import pytest

import paper_2106_12270_gb300 as wrs
from paper_2106_12270_gb300 import _build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fname in os.listdir(os.path.join(ROOT, "include")):
        if not fname.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fname)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w \t\*]*?\b(wrs_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return wrs.lib()


def test_header_declares_entry_points():
    names = declared_functions()
    for must in ("wrs_build_rows", "wrs_sample_rows", "wrs_step_total", "wrs_step_partition",
                 "wrs_step_split", "wrs_step_pack", "wrs_strerror"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    raw = ctypes.CDLL(_build.LIB)
    missing = [n for n in declared_functions() if not hasattr(raw, n)]
    assert not missing, missing


def test_host_argument_checks(lib):
    out = ctypes.c_uint64()
    assert lib.wrs_build_workspace_bytes(0, None, ctypes.byref(out)) == wrs.EINVAL
    assert lib.wrs_build_workspace_bytes(2**31, None, ctypes.byref(out)) == wrs.EINVAL
    assert lib.wrs_build_workspace_bytes(1000, None, ctypes.byref(out)) == wrs.OK
    assert out.value > 8 * 1000
    bad = wrs.config(section_size=300)
    assert lib.wrs_build_workspace_bytes(1000, ctypes.byref(bad), ctypes.byref(out)) == wrs.EINVAL
    bad = wrs.config(split_method=9)
    assert lib.wrs_build_workspace_bytes(1000, ctypes.byref(bad), ctypes.byref(out)) == wrs.EINVAL
    # null pointers are rejected before anything is enqueued
    assert lib.wrs_build_rows(None, 10, None, None, 0, None, None, None) == wrs.EINVAL
    assert lib.wrs_sample_rows(None, 10, 0, 5, 1, 0, 0, None, None) == wrs.EINVAL
    assert lib.wrs_sample_rows(None, 0, 0, 5, 1, 0, 0, None, None) == wrs.EINVAL
    # the Philox probe needs an 8-byte aligned output (checked on the host)
    assert lib.wrs_diag_philox(4, 1, ctypes.c_void_p(4), None) == wrs.EINVAL
    assert lib.wrs_diag_philox(4, 1, None, None) == wrs.EINVAL
    # pack variants: a missing workspace, then an unknown variant (a fake,
    # never dereferenced workspace address passes the workspace checks)
    big = 1 << 40
    assert lib.wrs_diag_pack_variant(None, 10, None, None, 0, None, 1, None) == wrs.EINVAL
    assert lib.wrs_diag_pack_variant(None, 10, ctypes.c_void_p(256), ctypes.c_void_p(256), big,
                                     None, 3, None) == wrs.EINVAL
    assert lib.wrs_diag_pack_variant(None, 10, ctypes.c_void_p(256), ctypes.c_void_p(256), big,
                                     None, 0, None) == wrs.EINVAL   # gather needs the weights
    # PSA+: a missing or misaligned workspace
    assert lib.wrs_build_rows_plus(None, 10, None, None, 0, None, 1, None, None, None) == wrs.EINVAL
    assert lib.wrs_build_rows_plus(ctypes.c_void_p(256), 10, ctypes.c_void_p(256),
                                   ctypes.c_void_p(100), big, None, 1, ctypes.c_void_p(256),
                                   None, None) == wrs.EINVAL
    assert lib.wrs_abi_version() >= 1
    assert lib.wrs_strerror(wrs.EZEROSUM) == b"all weights are zero"


def test_handle_calls_check_arguments_on_the_host(lib):
    P = ctypes.c_void_p
    h = P()
    # build(weights) -> table: bad sizes and pointers fail before any CUDA call
    assert lib.wrs_build(None, 10, 1, None, ctypes.byref(h)) == wrs.EINVAL
    assert lib.wrs_build(P(256), 0, 1, None, ctypes.byref(h)) == wrs.EINVAL
    assert lib.wrs_build(P(256), 2**31, 1, None, ctypes.byref(h)) == wrs.EINVAL
    assert lib.wrs_build(P(258), 10, 1, None, ctypes.byref(h)) == wrs.EINVAL   # misaligned
    assert lib.wrs_build(P(256), 10, 1, None, None) == wrs.EINVAL
    assert h.value is None
    assert lib.wrs_sample(None, 5, 1, P(256), wrs.SAMPLE_NAIVE, None) == wrs.EINVAL
    assert lib.wrs_table_info(None, None, None, None, None) == wrs.EINVAL
    assert lib.wrs_table_export(None, P(256), 0) == wrs.EINVAL
    assert lib.wrs_table_import(None, 10, 0, 1.0, ctypes.byref(h)) == wrs.EINVAL
    assert lib.wrs_table_destroy(None) == wrs.OK
    assert lib.wrs_build_batched(None, None, 3, None, ctypes.byref(h)) == wrs.EINVAL
    assert lib.wrs_build_batched(P(256), P(256), 0, None, ctypes.byref(h)) == wrs.EINVAL
    assert lib.wrs_batch_status(None, None) == wrs.EINVAL
    assert lib.wrs_sample_batched(None, P(256), 1, P(256), None) == wrs.EINVAL
    assert lib.wrs_batch_destroy(None) == wrs.OK
    # process-wide build settings: checked like a per-call config
    cur = wrs.Config()
    assert lib.wrs_get_config(ctypes.byref(cur)) == wrs.OK
    assert lib.wrs_set_config(ctypes.byref(wrs.config(section_size=300))) == wrs.EINVAL
    after = wrs.Config()
    lib.wrs_get_config(ctypes.byref(after))
    assert after.section_size == cur.section_size
    # measurement calls
    assert lib.wrs_diag_random_gather(P(256), 10, 5, 1, 0, 0, 8, P(256), None) == wrs.EINVAL
    assert lib.wrs_diag_random_gather(P(256), 10, 5, 1, 0, 8, 3, P(256), None) == wrs.EINVAL
    assert lib.wrs_diag_random_gather(P(256), 10, 5, 1, 3, 8, 8, P(256), None) == wrs.EINVAL
    assert lib.wrs_diag_build_each(None, None, 3, None, None, 0, None, None, None) == wrs.EINVAL


def test_noalloc_array_holds_the_largest_accepted_build(lib):
    # the allocation-free build accepts n <= 3.5 million with any section
    # size; its workspace is a 32 MiB array, and the layout is largest for
    # the smallest sections
    out = ctypes.c_uint64()
    for sec in (256, 1024, 8192):
        c = wrs.config(section_size=sec)
        assert lib.wrs_build_workspace_bytes(3_500_000, ctypes.byref(c), ctypes.byref(out)) == wrs.OK
        assert out.value <= 32 << 20, (sec, out.value)


def test_layout_is_aligned_and_ordered(lib):
    for n in (1, 31, 4096, 10**6 + 3):
        L = wrs.build_layout(n)
        offs = [L["lh"], L["ckl"], L["ckh"], L["splits"]]
        assert all(o % 256 == 0 for o in offs)
        assert offs == sorted(offs) and offs[-1] < L["total_bytes"]
        assert L["ckl"] - L["lh"] >= 8 * n
        assert L["sections"] == (n + 1023) // 1024
        assert wrs.build_workspace_bytes(n) == L["total_bytes"]
