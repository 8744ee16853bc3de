"""CPU oracle for GTS range / kNN search -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` import this package.  The library (``paper_2404_00966_gb300``)
never imports, links or executes it, and the two share no code: the only
common module is ``synth`` (seeded inputs, no method arithmetic).

``oracle.c`` holds the plain definitions (brute force over every visible
object, FP64 or integer metric; Section 3, Definitions 1 and 2).  ``index.py``
holds Algorithms 1-3 (index construction) written step by step in numpy.
The multi-column functions at the end define the summed distance of the
closing remark of Section 5.2 and answer its queries by brute force.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess

import numpy as np

from synth import Strings

EDIT, L1, L2, COS = 0, 1, 2, 3
METRICS = {"edit": EDIT, "l1": L1, "l2": L2, "cos": COS}

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c with gcc (-O2, OpenMP, no FP contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fPIC",
                               "-shared", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        I64 = ctypes.c_int64
        L.orc_threads.restype = ctypes.c_int
        L.orc_edit_full.restype = I64
        L.orc_edit_full.argtypes = [P, I64, P, I64]
        L.orc_edit_banded.restype = I64
        L.orc_edit_banded.argtypes = [P, I64, P, I64, I64]
        L.orc_l2sq.restype = ctypes.c_double
        L.orc_l2sq.argtypes = [P, P, I64]
        L.orc_l1.restype = ctypes.c_double
        L.orc_l1.argtypes = [P, P, I64]
        L.orc_cos_key.restype = ctypes.c_double
        L.orc_cos_key.argtypes = [P, P, I64]
        L.orc_cos_limit.restype = ctypes.c_double
        L.orc_cos_limit.argtypes = [ctypes.c_double]
        L.orc_cos_angles.argtypes = [P, I64, P]
        L.orc_keys_vec.argtypes = [ctypes.c_int, P, I64, I64, P, P]
        L.orc_keys_str.argtypes = [P, P, I64, P, I64, P]
        L.orc_range_vec.argtypes = [ctypes.c_int, P, I64, I64, P, I64, P, P, P, P, P, P, P, P]
        L.orc_range_str.argtypes = [P, P, I64, P, P, I64, P, P, P, P, P, P, P, P]
        L.orc_knn_vec.argtypes = [ctypes.c_int, P, I64, I64, P, I64, P, P, P, P, P, P, P, P]
        L.orc_knn_str.argtypes = [P, P, I64, P, P, I64, P, P, P, P, P, P, P, P]
        _lib = L
    return _lib


def threads() -> int:
    return int(lib().orc_threads())


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


# ------------------------------------------------------------------ metrics

def edit_full(a: bytes, b: bytes) -> int:
    A = np.frombuffer(a, np.uint8) if len(a) else np.zeros(1, np.uint8)
    B = np.frombuffer(b, np.uint8) if len(b) else np.zeros(1, np.uint8)
    return int(lib().orc_edit_full(_p(A), len(a), _p(B), len(b)))


def edit_banded(a: bytes, b: bytes, r: int) -> int:
    A = np.frombuffer(a, np.uint8) if len(a) else np.zeros(1, np.uint8)
    B = np.frombuffer(b, np.uint8) if len(b) else np.zeros(1, np.uint8)
    return int(lib().orc_edit_banded(_p(A), len(a), _p(B), len(b), int(r)))


def l2sq(a, b) -> float:
    a = np.ascontiguousarray(a, np.float32)
    b = np.ascontiguousarray(b, np.float32)
    return float(lib().orc_l2sq(_p(a), _p(b), a.shape[0]))


def l1(a, b) -> float:
    a = np.ascontiguousarray(a, np.float32)
    b = np.ascontiguousarray(b, np.float32)
    return float(lib().orc_l1(_p(a), _p(b), a.shape[0]))


def cos_key(a, b) -> float:
    """1 - cos of the angle between two vectors (FP64 sums, c clamped)."""
    a = np.ascontiguousarray(a, np.float32)
    b = np.ascontiguousarray(b, np.float32)
    return float(lib().orc_cos_key(_p(a), _p(b), a.shape[0]))


def cos_limit(r: float) -> float:
    """The range limit on the key for an angle r: 1 - cos(min(r, pi))."""
    return float(lib().orc_cos_limit(float(np.float32(r))))


def keys_to_pivot(metric: str, objects, pivot_index: int) -> np.ndarray:
    """Exact keys (FP64 for vectors: d^2 for L2, d for L1; int for edit) from
    object ``pivot_index`` to every object."""
    m = METRICS[metric]
    if m == EDIT:
        S: Strings = objects
        out = np.empty(S.n, np.int64)
        q = np.ascontiguousarray(S.data[S.offsets[pivot_index]:S.offsets[pivot_index + 1]])
        if q.shape[0] == 0:
            q = np.zeros(1, np.uint8)
        lq = int(S.offsets[pivot_index + 1] - S.offsets[pivot_index])
        data = S.data if S.data.shape[0] else np.zeros(1, np.uint8)
        lib().orc_keys_str(_p(data), _p(S.offsets), S.n, _p(q), lq, _p(out))
        return out
    X = np.ascontiguousarray(objects, np.float32)
    out = np.empty(X.shape[0], np.float64)
    lib().orc_keys_vec(m, _p(X), X.shape[0], X.shape[1], _p(np.ascontiguousarray(X[pivot_index])), _p(out))
    return out


def distances_to(metric: str, objects, target) -> np.ndarray:
    """FP64 (or integer) distance from ``target`` to every object."""
    m = METRICS[metric]
    if m == EDIT:
        S: Strings = objects
        q = np.frombuffer(target, np.uint8) if len(target) else np.zeros(1, np.uint8)
        out = np.empty(S.n, np.int64)
        data = S.data if S.data.shape[0] else np.zeros(1, np.uint8)
        lib().orc_keys_str(_p(data), _p(S.offsets), S.n, _p(q), len(target), _p(out))
        return out.astype(np.float64)
    X = np.ascontiguousarray(objects, np.float32)
    t = np.ascontiguousarray(target, np.float32)
    out = np.empty(X.shape[0], np.float64)
    lib().orc_keys_vec(m, _p(X), X.shape[0], X.shape[1], _p(t), _p(out))
    return key_to_distance(metric, out)


def key_to_distance(metric: str, keys: np.ndarray) -> np.ndarray:
    if metric == "l2":
        return np.sqrt(keys)
    if metric == "cos":
        return np.arccos(1.0 - keys)
    return keys


# ------------------------------------------------------------------ queries

def _seq_args(ins_seq, del_seq, qseq):
    if ins_seq is None:
        return None, None, None
    return (np.ascontiguousarray(ins_seq, np.int64), np.ascontiguousarray(del_seq, np.int64),
            np.ascontiguousarray(qseq, np.int64))


def range_query(metric: str, objects, queries, radii, ins_seq=None, del_seq=None, qseq=None):
    """Brute-force MRQ for every query (Definition 1).  Returns CSR
    ``(offsets int64[nq+1], ids int64[], dist float64[])``, ids ascending per
    query.  ``dist`` is sqrt(key) for L2, the key for L1 and edit."""
    m = METRICS[metric]
    radii = np.ascontiguousarray(radii, np.float32)
    ins, dele, qs = _seq_args(ins_seq, del_seq, qseq)
    L = lib()
    if m == EDIT:
        S: Strings = objects
        Qs: Strings = queries
        nq = Qs.n
        counts = np.zeros(nq, np.int64)
        sd = S.data if S.data.shape[0] else np.zeros(1, np.uint8)
        qd = Qs.data if Qs.data.shape[0] else np.zeros(1, np.uint8)
        args = (_p(sd), _p(S.offsets), S.n, _p(qd), _p(Qs.offsets), nq, _p(radii), _p(ins), _p(dele), _p(qs))
        L.orc_range_str(*args, _p(counts), None, None, None)
        offsets = np.zeros(nq + 1, np.int64)
        np.cumsum(counts, out=offsets[1:])
        ids = np.empty(max(1, int(offsets[-1])), np.int64)
        keys = np.empty(max(1, int(offsets[-1])), np.float64)
        L.orc_range_str(*args, _p(counts), _p(offsets), _p(ids), _p(keys))
    else:
        X = np.ascontiguousarray(objects, np.float32)
        Q = np.ascontiguousarray(queries, np.float32)
        nq = Q.shape[0]
        counts = np.zeros(nq, np.int64)
        args = (m, _p(X), X.shape[0], X.shape[1], _p(Q), nq, _p(radii), _p(ins), _p(dele), _p(qs))
        L.orc_range_vec(*args, _p(counts), None, None, None)
        offsets = np.zeros(nq + 1, np.int64)
        np.cumsum(counts, out=offsets[1:])
        ids = np.empty(max(1, int(offsets[-1])), np.int64)
        keys = np.empty(max(1, int(offsets[-1])), np.float64)
        L.orc_range_vec(*args, _p(counts), _p(offsets), _p(ids), _p(keys))
    tot = int(offsets[-1])
    ids, keys = ids[:tot], keys[:tot]
    return offsets, ids, key_to_distance(metric, keys), keys


def knn_query(metric: str, objects, queries, k, ins_seq=None, del_seq=None, qseq=None):
    """Brute-force MkNNQ (Definition 2): per query the first min(k, visible)
    objects in ascending (key, id) order.  Returns CSR
    ``(offsets, ids, dist, keys)``."""
    m = METRICS[metric]
    ins, dele, qs = _seq_args(ins_seq, del_seq, qseq)
    L = lib()
    nq = queries.n if m == EDIT else int(np.asarray(queries).shape[0])
    k = np.ascontiguousarray(np.broadcast_to(np.asarray(k, np.int32), (nq,)), np.int32)
    cap = np.zeros(nq + 1, np.int64)
    np.cumsum(k.astype(np.int64), out=cap[1:])
    ids = np.empty(max(1, int(cap[-1])), np.int64)
    keys = np.empty(max(1, int(cap[-1])), np.float64)
    counts = np.zeros(nq, np.int64)
    if m == EDIT:
        S: Strings = objects
        Qs: Strings = queries
        sd = S.data if S.data.shape[0] else np.zeros(1, np.uint8)
        qd = Qs.data if Qs.data.shape[0] else np.zeros(1, np.uint8)
        L.orc_knn_str(_p(sd), _p(S.offsets), S.n, _p(qd), _p(Qs.offsets), nq, _p(k), _p(ins), _p(dele),
                      _p(qs), _p(cap), _p(ids), _p(keys), _p(counts))
    else:
        X = np.ascontiguousarray(objects, np.float32)
        Q = np.ascontiguousarray(queries, np.float32)
        L.orc_knn_vec(m, _p(X), X.shape[0], X.shape[1], _p(Q), nq, _p(k), _p(ins), _p(dele), _p(qs),
                      _p(cap), _p(ids), _p(keys), _p(counts))
    offsets = np.zeros(nq + 1, np.int64)
    np.cumsum(counts, out=offsets[1:])
    sel = np.concatenate([np.arange(cap[i], cap[i] + counts[i]) for i in range(nq)]) if nq else np.zeros(0, np.int64)
    sel = sel.astype(np.int64)
    return offsets, ids[sel], key_to_distance(metric, keys[sel]), keys[sel]


# ------------------------------------------------------------ multi-column

def column_distances(metric: str, objects, target) -> np.ndarray:
    """FP64 column distance from ``target`` to every object for a
    multi-column query: sqrt of the FP64 key for L2, the key for L1, and for
    the angle the C library's acos of 1 - key (the function Python's
    ``math.acos`` calls, run in a C loop)."""
    m = METRICS[metric]
    if m == EDIT:
        raise ValueError("multi-column queries take vector columns")
    X = np.ascontiguousarray(objects, np.float32)
    t = np.ascontiguousarray(target, np.float32)
    keys = np.empty(X.shape[0], np.float64)
    lib().orc_keys_vec(m, _p(X), X.shape[0], X.shape[1], _p(t), _p(keys))
    if metric == "l2":
        return np.sqrt(keys)
    if metric == "cos":
        out = np.empty_like(keys)
        lib().orc_cos_angles(_p(keys), keys.shape[0], _p(out))
        return out
    return keys


def multi_sums(metrics, columns, queries, qi: int) -> np.ndarray:
    """Distance of every object from query ``qi`` over several columns (the
    closing remark of Section 5.2): the column distances summed in column
    order in FP64, starting from 0."""
    s = np.zeros(np.asarray(columns[0]).shape[0], np.float64)
    for metric, X, Q in zip(metrics, columns, queries):
        s = s + column_distances(metric, X, np.asarray(Q)[qi])
    return s


def multi_range(metrics, columns, queries, radii, live=None):
    """Brute-force multi-column MRQ (Definition 1 over the summed distance):
    per query every live object whose sum is <= r, ascending id.  ``live``:
    optional bool mask over the ids.  Returns ``(offsets, ids, sums)``."""
    nq = int(np.asarray(queries[0]).shape[0])
    radii = np.asarray(radii, np.float32)
    offsets, ids, sums = [0], [], []
    for q in range(nq):
        s = multi_sums(metrics, columns, queries, q)
        keep = s <= float(radii[q])
        if live is not None:
            keep &= live
        sel = np.nonzero(keep)[0]
        ids.append(sel)
        sums.append(s[sel])
        offsets.append(offsets[-1] + sel.shape[0])
    cat = (lambda a, t: np.concatenate(a).astype(t) if a else np.zeros(0, t))
    return np.asarray(offsets, np.int64), cat(ids, np.int64), cat(sums, np.float64)


def multi_knn(metrics, columns, queries, k, live=None):
    """Brute-force multi-column MkNNQ (Definition 2 over the summed
    distance): per query the first min(k, live objects) in ascending
    (sum, id) order.  Returns ``(offsets, ids, sums)``."""
    nq = int(np.asarray(queries[0]).shape[0])
    k = np.broadcast_to(np.asarray(k, np.int64), (nq,))
    offsets, ids, sums = [0], [], []
    for q in range(nq):
        s = multi_sums(metrics, columns, queries, q)
        cand = np.arange(s.shape[0]) if live is None else np.nonzero(live)[0]
        order = cand[np.lexsort((cand, s[cand]))][: int(k[q])]
        ids.append(order)
        sums.append(s[order])
        offsets.append(offsets[-1] + order.shape[0])
    cat = (lambda a, t: np.concatenate(a).astype(t) if a else np.zeros(0, t))
    return np.asarray(offsets, np.int64), cat(ids, np.int64), cat(sums, np.float64)
