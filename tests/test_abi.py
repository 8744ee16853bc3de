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


@pytest.mark.skipif(os.path.exists("/dev/nvidia0"), reason="a GPU is present")
def test_no_device_means_an_error_not_a_fallback(L):
    import paper_2404_00966_gb300 as g
    X = np.random.default_rng(0).random((50, 4), dtype=np.float32)
    with pytest.raises(g.GTSError) as e:
        g.Index.build(X, "l2", fanout=4)
    assert e.value.name == "GTS_ECUDA"
