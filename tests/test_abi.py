"""The C-ABI library loads and exports every entry point that include/gts.h
declares; without a device every call fails loudly (no CPU fallback).  CPU
only: no compute call reaches a GPU here."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gts.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gts_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def L():
    from paper_2404_00966_gb300 import build_ext
    build_ext.build()
    import paper_2404_00966_gb300 as g
    return g.lib()


def test_header_declares_the_boundary():
    names = _declared()
    for f in ["gts_build", "gts_range", "gts_knn", "gts_insert", "gts_delete", "gts_batch_update",
              "gts_result_free", "gts_free", "gts_last_error"]:
        assert f in names


def test_library_exports_every_declared_symbol(L):
    missing = [f for f in _declared() if not hasattr(L, f)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    import paper_2404_00966_gb300 as g
    assert sorted(g.EXPORTS) == _declared()


def test_status_names(L):
    names = [L.gts_status_name(i).decode() for i in range(7)]
    assert names == ["GTS_OK", "GTS_EINVAL", "GTS_ENOMEM", "GTS_ECUDA", "GTS_ETIMEOUT", "GTS_ENOTFOUND",
                     "GTS_EOVERFLOW"]


def test_argument_errors_are_reported_before_any_device_work(L):
    import paper_2404_00966_gb300 as g
    out = ctypes.c_void_p()
    # metric / object mismatch, bad fanout: rejected by argument checks
    X = np.zeros((4, 3), np.float32)
    o = g._Objects(n=4, dim=3, on_device=0, data=X.ctypes.data, offsets=None)
    assert L.gts_build(ctypes.byref(o), g.EDIT, 0, 8, None, ctypes.byref(out)) == 1
    assert b"strings" in L.gts_last_error()
    assert L.gts_build(ctypes.byref(o), g.L2, 0, 1, None, ctypes.byref(out)) == 1
    assert L.gts_build(ctypes.byref(o), 7, 0, 8, None, ctypes.byref(out)) == 1


def test_multi_column_argument_errors_without_a_device(L):
    import paper_2404_00966_gb300 as g
    res = g._Result()
    assert L.gts_multi_range(None, 1, None, None, None, ctypes.byref(res)) == 1
    assert b"NULL" in L.gts_last_error()
    hs = (ctypes.c_void_p * 1)(None)
    q = (g._Objects * 1)()
    assert L.gts_multi_knn(hs, 0, q, None, None, ctypes.byref(res)) == 1
    assert b"columns" in L.gts_last_error()
    assert L.gts_multi_knn(hs, 1, q, None, None, ctypes.byref(res)) == 1


@pytest.mark.skipif(os.path.exists("/dev/nvidia0"), reason="a GPU is present")
def test_no_device_means_an_error_not_a_fallback(L):
    import paper_2404_00966_gb300 as g
    X = np.random.default_rng(0).random((50, 4), dtype=np.float32)
    with pytest.raises(g.GTSError) as e:
        g.Index.build(X, "l2", fanout=4)
    assert e.value.name == "GTS_ECUDA"


def test_cost_model_closed_form(L):
    """gts_cost_model (Section 5.3) is host arithmetic: S_i = nq (F p)^i per
    pivot level, S_{h+1} = nq n p^h for the objects of the surviving leaves,
    cost = sum_i i^2 ceil(S_i / C) log2(F)^2.  Worked by hand for n = 1000,
    nq = 10, p = 1/2, F = 4, h = 2, C = 8:
    level 1: S = 20, ceil(20/8) = 3, 1 * 3 * 4 = 12;
    level 2: S = 40, ceil(40/8) = 5, 4 * 5 * 4 = 80;
    leaves:  S = 2500, ceil(2500/8) = 313, 9 * 313 * 4 = 11268; total 11360."""
    import paper_2404_00966_gb300 as g
    assert g.cost_model(1000, 10, 0.5, 4, 2, 8.0) == 11360.0
    # nothing survives the first pivot level: no work anywhere
    assert g.cost_model(1000, 10, 0.0, 4, 3, 8.0) == 0.0
    # p = 1 (no pruning) with h = 1, F = 2: level 10 * 2 = 20 -> 3 * 1;
    # leaves 10 * 1000 = 10000 -> 1250 * 4; log2(2)^2 = 1
    assert g.cost_model(1000, 10, 1.0, 2, 1, 8.0) == 3.0 + 4 * 1250.0
    # arguments out of range give -1
    for bad in [(1000, 10, 1.5, 4, 2, 8.0), (1000, 10, 0.5, 1, 2, 8.0), (1000, 10, 0.5, 4, 0, 8.0),
                (1000, 10, 0.5, 4, 2, 0.0)]:
        assert g.cost_model(*bad) == -1.0
