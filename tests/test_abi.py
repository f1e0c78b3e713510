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


def test_layout_is_aligned_and_ordered(lib):
    for n in (1, 31, 4096, 10**6 + 3):
        L = wrs.build_layout(n)
        offs = [L["lh"], L["ckl"], L["ckh"], L["splits"]]
        assert all(o % 256 == 0 for o in offs)
        assert offs == sorted(offs) and offs[-1] < L["total_bytes"]
        assert L["ckl"] - L["lh"] >= 8 * n
        assert L["sections"] == (n + 1023) // 1024
        assert wrs.build_workspace_bytes(n) == L["total_bytes"]
