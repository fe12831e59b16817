"""C-ABI checks that need no GPU: the library builds for sm_103a, loads, exports every
entry point declared in include/tmc.h, and rejects malformed descriptions before any
device work."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_1806_08593_gb300 import tmc
from paper_1806_08593_gb300.build import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build()
    return tmc.load_library()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "tmc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(tmc_[a-z_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert "tmc_plan_create" in names and "tmc_backward" in names
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) == set(tmc.EXPORTS)


def test_status_strings(lib):
    for code, name in tmc.STATUS.items():
        assert lib.tmc_status_string(code).decode() == name


def _desc(n, parent, K, d, obs, shared=0, pv=1.0, ov=0.1, prec=0):
    arrs = [np.ascontiguousarray(a, dtype=np.int32) for a in (n, parent, K, d, obs)]
    desc = tmc.ProblemDesc(len(arrs[0]), *[a.ctypes.data for a in arrs], shared, pv, ov, prec)
    return desc, arrs


@pytest.mark.parametrize("case", [
    dict(n=[3], parent=[0, 0, 1], K=[4], d=[2], obs=[2]),          # root parent not -1
    dict(n=[3], parent=[-1, 2, 0], K=[4], d=[2], obs=[2]),         # parent after child
    dict(n=[2], parent=[-1, 0], K=[0], d=[2], obs=[2]),            # K = 0
    dict(n=[2], parent=[-1, 0], K=[4], d=[0], obs=[2]),            # d = 0
    dict(n=[0], parent=[], K=[4], d=[2], obs=[2]),                 # empty instance
    dict(n=[2], parent=[-1, 0], K=[4], d=[2], obs=[2], pv=0.0),    # zero variance
    dict(n=[2], parent=[-1, 0], K=[4], d=[2], obs=[2], prec=9),    # unknown precision
    dict(n=[2], parent=[-1, 0], K=[4], d=[2], obs=[2], prec=1),    # reserved (no bf16 path)
    dict(n=[2, 3], parent=[-1, 0, -1, 0, 0], K=[4, 4], d=[2, 2], obs=[2, 2], shared=1),  # shared mismatch
])
def test_invalid_descriptions_rejected(lib, case):
    desc, keep = _desc(case["n"], case["parent"] or [0], case["K"], case["d"], case["obs"],
                       case.get("shared", 0), case.get("pv", 1.0), 0.1, case.get("prec", 0))
    h = ctypes.c_void_p()
    st = lib.tmc_plan_create(ctypes.byref(desc), ctypes.byref(h))
    assert st == 1 and not h.value


def test_unsupported_sizes_rejected(lib):
    desc, keep = _desc([2], [-1, 0], [20000], [2], [2])
    h = ctypes.c_void_p()
    assert lib.tmc_plan_create(ctypes.byref(desc), ctypes.byref(h)) == 2
    desc, keep = _desc([2], [-1, 0], [4], [2000], [2])
    assert lib.tmc_plan_create(ctypes.byref(desc), ctypes.byref(h)) == 2


def test_null_arguments(lib):
    h = ctypes.c_void_p()
    assert lib.tmc_plan_create(None, ctypes.byref(h)) == 1
    assert lib.tmc_log_marginal(None, None, None, None) == 1
    assert lib.tmc_backward(None, None, None, None, None) == 1
    assert lib.tmc_plan_destroy(None) == 0
    assert lib.tmc_plan_sync_status(None, None) == 1


def test_alloc_fault_is_reported(lib, monkeypatch):
    """TMC_FAULT=alloc: plan creation fails as if the workspace allocation had, before any
    device allocation (so this runs without a GPU)."""
    monkeypatch.setenv("TMC_FAULT", "alloc")
    desc, keep = _desc([3], [-1, 0, 1], [4], [2], [2])
    h = ctypes.c_void_p()
    assert lib.tmc_plan_create(ctypes.byref(desc), ctypes.byref(h)) == 3
    assert not h.value


def test_wait_limit_arguments(lib):
    assert lib.tmc_plan_set_wait_limit(None, 1 << 20) == 1
