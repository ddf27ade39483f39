"""The C-ABI library builds for sm_103a, loads, and exports every symbol bbc.h declares.

These run without a GPU: they call no entry point that touches the device.
"""

from __future__ import annotations

import ctypes
import os
import re
import subprocess

import pytest

from paper_2601_17707_gb300 import _build, bbc

HEADER = os.path.join(_build.ROOT, "include", "bbc.h")


def declared_functions() -> list[str]:
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(bbc_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return bbc.load()


def test_header_and_binding_agree():
    assert declared_functions() == sorted(bbc.EXPORTS)


def test_build_targets_sm_103a_only():
    assert _build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", _build.LIB], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\bT (bbc_[a-z_0-9]+)$", out, flags=re.M))
    assert set(declared_functions()) <= exported


def test_status_strings(lib):
    for code, name in bbc.STATUS_NAMES.items():
        s = lib.bbc_status_string(code)
        assert isinstance(s, bytes) and s
    assert lib.bbc_status_string(999) == b"unknown status"


def test_tuning_defaults_are_host_only(lib):
    t = bbc.default_tuning()
    assert t.tile_words > 0 and t.tile_words % 8 == 0
    assert 0 < t.warp_max_wedges <= 512
    assert t.blocks_per_sm in (1, 2)


def test_invalid_arguments_are_rejected_before_any_device_work(lib):
    h = ctypes.c_void_p()
    assert lib.bbc_prepare(-1, 2, 0, None, None, None, 0, None, ctypes.byref(h)) == 1
    assert lib.bbc_prepare(2, 2, 3, None, None, None, 0, None, ctypes.byref(h)) == 1
    assert lib.bbc_prepare(2, 2, 0, None, None, None, 4 | 8, None, ctypes.byref(h)) == 1
    assert b"both side flags" in lib.bbc_last_error()
    b = ctypes.c_uint64()
    assert lib.bbc_count(None, ctypes.byref(b), None, None, None, None, None) == 1
    out = (ctypes.c_uint64 * 6)()
    assert lib.bbc_count_motif(None, 1, 2, ctypes.addressof(out), None) == 1
    assert b"bbc_count_motif" in lib.bbc_last_error()
    d = ctypes.c_int64()
    assert lib.bbc_count_delta(None, 0, None, None, None, 0, ctypes.byref(d), None, None) == 1
    assert lib.bbc_graph_work(None, ctypes.addressof(out), None) == 1
    assert lib.bbc_cost_model_create(0, None) == 1
    assert lib.bbc_cost_model_get_params(None, None, 0) == 1
    assert lib.bbc_cost_model_order(None, None, None) == 1
    assert lib.bbc_item_features(None, None, 0, None, None) == 1
    n_items = ctypes.c_int32()
    assert lib.bbc_item_anchors(None, None, 0, ctypes.byref(n_items), None) == 1
    assert b"bbc_item_anchors" in lib.bbc_last_error()
    assert lib.bbc_cost_model_num_params() == 1377
    lib.bbc_cost_model_free(None)
    lib.bbc_graph_free(None)
