"""Python binding of the GTS C ABI (include/gts.h): exact batched metric range
and kNN search on a GB300 over a GTS index (arXiv 2404.00966).

Argument marshalling only: every step of the search runs in the CUDA library
``_build/libgts.so``.  There is no CPU fallback -- if the library is missing
or no device is usable, every call raises :class:`GTSError`.

Inputs may be numpy arrays (host) or torch CUDA tensors (device):
  * vectors: float32 ``[n, dim]``;
  * strings: ``synth.Strings`` (host) or a pair ``(bytes uint8, offsets int64)``
    of numpy arrays or of CUDA tensors.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

__all__ = ["GTSError", "Index", "ShardedIndex", "Server", "lib", "merge_knn", "merge_range", "cost_model", "EDIT",
           "L1", "L2", "COS", "PREC_FP32", "PREC_BF16", "STAT_NAMES"]

EDIT, L1, L2, COS = 0, 1, 2, 3
PREC_FP32, PREC_BF16 = 0, 1
QUERY_COUNT_TABLE_PASS, QUERY_KEYS = 1, 2
METRIC_IDS = {"edit": EDIT, "l1": L1, "l2": L2, "cos": COS}
STAT_NAMES = ["pivot_dist", "frontier", "scanned_rows", "candidates", "rechecks", "results", "groups", "cache_rows",
              "launches", "tiles", "tile_entries", "tile_pairs",
              "dense_pairs", "dense_last", "table_pass", "scan_records"]
STAGE_NAMES = ["pivot_dist", "threshold", "expand", "leaf_scan", "verify", "select", "other", "tile"]

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libgts.so")
_lib = None


class GTSError(RuntimeError):
    def __init__(self, status: int, name: str, msg: str):
        super().__init__(f"{name}: {msg}")
        self.status = status
        self.name = name


class _Objects(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("dim", ctypes.c_int32), ("on_device", ctypes.c_int32),
                ("data", ctypes.c_void_p), ("offsets", ctypes.c_void_p)]


class _BuildOpts(ctypes.Structure):
    _fields_ = [("stream", ctypes.c_void_p), ("root_pivot", ctypes.c_int64), ("seed", ctypes.c_uint64),
                ("cache_limit", ctypes.c_int64)]


class _QueryOpts(ctypes.Structure):
    _fields_ = [("stream", ctypes.c_void_p), ("precision", ctypes.c_int32), ("result_on_device", ctypes.c_int32),
                ("memory_budget", ctypes.c_int64), ("seq", ctypes.c_void_p), ("stats", ctypes.c_void_p),
                ("stage_ms", ctypes.c_void_p), ("flags", ctypes.c_int32), ("reserved_", ctypes.c_int32)]


class _Result(ctypes.Structure):
    _fields_ = [("nq", ctypes.c_int64), ("offsets", ctypes.c_void_p), ("ids", ctypes.c_void_p),
                ("dist", ctypes.c_void_p), ("on_device", ctypes.c_int32), ("priv_", ctypes.c_void_p),
                ("key", ctypes.c_void_p)]


class _ServeOpts(ctypes.Structure):
    _fields_ = [("max_batch", ctypes.c_int32), ("n_streams", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("batch_quantum", ctypes.c_int32), ("result_budget", ctypes.c_int64),
                ("memory_budget", ctypes.c_int64)]


class _Info(ctypes.Structure):
    _fields_ = [("n_tree", ctypes.c_int64), ("n_cache", ctypes.c_int64), ("n_live", ctypes.c_int64),
                ("next_id", ctypes.c_int64), ("seq", ctypes.c_int64), ("rebuild_seq", ctypes.c_int64),
                ("h", ctypes.c_int32), ("fanout", ctypes.c_int32), ("metric", ctypes.c_int32),
                ("dim", ctypes.c_int32), ("device_bytes", ctypes.c_int64)]


class _Tuning(ctypes.Structure):
    _fields_ = [("l1_queries", ctypes.c_int32), ("l1_packed", ctypes.c_int32), ("knn_phases", ctypes.c_int32),
                ("probe_rows", ctypes.c_int32), ("tuned", ctypes.c_int32), ("tc_queries", ctypes.c_int32),
                ("str_chunk", ctypes.c_int32), ("str_qgram", ctypes.c_int32)]


TUNING_FIELDS = ["l1_queries", "l1_packed", "knn_phases", "probe_rows", "tc_queries", "str_chunk", "str_qgram"]


class _Shape(ctypes.Structure):
    _fields_ = [("fanout", ctypes.c_int32), ("n_pivots", ctypes.c_int32), ("model_cost", ctypes.c_double),
                ("measured_ms", ctypes.c_double)]

EXPORTS = ["gts_build", "gts_range", "gts_knn", "gts_insert", "gts_delete", "gts_batch_update", "gts_rebuild",
           "gts_info", "gts_tree_level", "gts_table", "gts_result_copy", "gts_result_free", "gts_free",
           "gts_last_error", "gts_status_name", "gts_selftest_tc", "gts_selftest_wait", "gts_knn_scan_noalloc",
           "gts_knn_scan_noalloc_async", "gts_serve_start",
           "gts_serve_submit", "gts_serve_wait", "gts_serve_stats", "gts_serve_project", "gts_serve_stop", "gts_get_tuning",
           "gts_set_tuning", "gts_autotune", "gts_cost_model", "gts_autotune_shape", "gts_save", "gts_load",
           "gts_merge_knn", "gts_merge_range", "gts_multi_range", "gts_multi_knn"]


def lib(path: Optional[str] = None):
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise GTSError(3, "GTS_ECUDA", f"CUDA library not built ({p}); run __graft_entry__.build()")
    L = ctypes.CDLL(p)
    P, I32, I64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    L.gts_build.argtypes = [ctypes.POINTER(_Objects), ctypes.c_int, ctypes.c_int, ctypes.c_int,
                            ctypes.POINTER(_BuildOpts), ctypes.POINTER(P)]
    L.gts_range.argtypes = [P, ctypes.POINTER(_Objects), P, ctypes.POINTER(_QueryOpts), ctypes.POINTER(_Result)]
    L.gts_knn.argtypes = [P, ctypes.POINTER(_Objects), P, ctypes.POINTER(_QueryOpts), ctypes.POINTER(_Result)]
    L.gts_insert.argtypes = [P, ctypes.POINTER(_Objects), P]
    L.gts_delete.argtypes = [P, P, I64, P]
    L.gts_batch_update.argtypes = [P, ctypes.POINTER(_Objects), P, I64, P]
    L.gts_rebuild.argtypes = [P]
    L.gts_info.argtypes = [P, ctypes.POINTER(_Info)]
    L.gts_tree_level.argtypes = [P, ctypes.c_int, P, P, P, P, P]
    L.gts_table.argtypes = [P, P, P]
    L.gts_serve_start.argtypes = [P, ctypes.POINTER(_ServeOpts), ctypes.POINTER(P)]
    L.gts_serve_submit.argtypes = [P, P, I64, I32, ctypes.c_double, ctypes.POINTER(I64)]
    L.gts_serve_wait.argtypes = [P, I64, I32, ctypes.POINTER(_Result), ctypes.POINTER(ctypes.c_double)]
    L.gts_serve_stats.argtypes = [P, P, I32]
    L.gts_serve_project.argtypes = [P, P, I64, I32, ctypes.c_double, P]
    L.gts_serve_stop.argtypes = [P]
    L.gts_get_tuning.argtypes = [P, ctypes.POINTER(_Tuning)]
    L.gts_set_tuning.argtypes = [P, ctypes.POINTER(_Tuning)]
    L.gts_autotune.argtypes = [P, ctypes.POINTER(_Objects), P, P, ctypes.POINTER(_QueryOpts), I32,
                               ctypes.POINTER(_Tuning)]
    for f in ["gts_serve_start", "gts_serve_submit", "gts_serve_wait", "gts_serve_stats", "gts_serve_stop",
              "gts_serve_project", "gts_get_tuning", "gts_set_tuning", "gts_autotune", "gts_autotune_shape"]:
        getattr(L, f).restype = ctypes.c_int
    for f in ["gts_knn_scan_noalloc", "gts_knn_scan_noalloc_async"]:
        getattr(L, f).argtypes = [P, I64, I32, ctypes.c_int, P, I64, I32, P, P, P]
        getattr(L, f).restype = ctypes.c_int
    L.gts_selftest_tc.argtypes = [P, P, ctypes.c_int, ctypes.c_int, ctypes.c_int, P]
    L.gts_selftest_tc.restype = ctypes.c_int
    L.gts_cost_model.argtypes = [I64, I64, ctypes.c_double, I32, I32, ctypes.c_double]
    L.gts_cost_model.restype = ctypes.c_double
    L.gts_autotune_shape.argtypes = [P, ctypes.POINTER(_Objects), P, P, ctypes.POINTER(_QueryOpts), I32, I32,
                                     ctypes.POINTER(_Shape), ctypes.POINTER(I32)]
    L.gts_save.argtypes = [P, ctypes.c_char_p]
    L.gts_load.argtypes = [ctypes.c_char_p, ctypes.POINTER(_BuildOpts), ctypes.POINTER(P)]
    L.gts_merge_knn.argtypes = [ctypes.POINTER(ctypes.POINTER(_Result)), P, I32, P, ctypes.POINTER(_Result)]
    L.gts_merge_range.argtypes = [ctypes.POINTER(ctypes.POINTER(_Result)), P, I32, ctypes.POINTER(_Result)]
    L.gts_multi_range.argtypes = [P, I32, ctypes.POINTER(_Objects), P, ctypes.POINTER(_QueryOpts),
                                  ctypes.POINTER(_Result)]
    L.gts_multi_knn.argtypes = [P, I32, ctypes.POINTER(_Objects), P, ctypes.POINTER(_QueryOpts),
                                ctypes.POINTER(_Result)]
    for f in ["gts_save", "gts_load", "gts_merge_knn", "gts_merge_range"]:
        getattr(L, f).restype = ctypes.c_int
    L.gts_selftest_wait.argtypes = [I32, ctypes.c_uint32]
    L.gts_selftest_wait.restype = ctypes.c_int
    L.gts_result_copy.argtypes = [ctypes.POINTER(_Result), P, P, P]
    L.gts_result_copy.restype = ctypes.c_int
    L.gts_result_free.argtypes = [ctypes.POINTER(_Result)]
    L.gts_result_free.restype = None
    L.gts_free.argtypes = [P]
    L.gts_free.restype = None
    L.gts_last_error.restype = ctypes.c_char_p
    L.gts_status_name.restype = ctypes.c_char_p
    L.gts_status_name.argtypes = [ctypes.c_int]
    for f in ["gts_build", "gts_range", "gts_knn", "gts_insert", "gts_delete", "gts_batch_update", "gts_rebuild",
              "gts_info", "gts_tree_level", "gts_table"]:
        getattr(L, f).restype = ctypes.c_int
    if path is None:
        _lib = L
    return L


def _host_arrays(res):
    nq = int(res.nq)
    offsets = np.ctypeslib.as_array(ctypes.cast(res.offsets, ctypes.POINTER(ctypes.c_int64)), (nq + 1,)).copy()
    tot = int(offsets[-1])
    ids = np.ctypeslib.as_array(ctypes.cast(res.ids, ctypes.POINTER(ctypes.c_int64)), (max(tot, 1),))[:tot].copy()
    dist = np.ctypeslib.as_array(ctypes.cast(res.dist, ctypes.POINTER(ctypes.c_float)), (max(tot, 1),))[:tot].copy()
    kk = None
    if res.key:
        kk = np.ctypeslib.as_array(ctypes.cast(res.key, ctypes.POINTER(ctypes.c_double)), (max(tot, 1),))[:tot].copy()
    return offsets, ids, dist, kk


def _c_result(offsets, ids, dist, keys=None):
    """A host gts_result viewing numpy arrays (kept alive by the caller)."""
    r = _Result()
    r.nq = int(len(offsets) - 1)
    r.offsets = _ptr(offsets).value
    r.ids = _ptr(ids).value if ids.size else _ptr(np.zeros(1, np.int64)).value
    r.dist = _ptr(dist).value if dist.size else _ptr(np.zeros(1, np.float32)).value
    r.on_device = 0
    r.priv_ = None
    r.key = _ptr(keys).value if keys is not None and keys.size else (
        _ptr(np.zeros(1, np.float64)).value if keys is not None else None)
    return r


def _merge(parts, id_base, k=None):
    """Merge host CSR answers of shards (gts_merge_knn / gts_merge_range).
    parts: (offsets, ids, dist[, keys]) tuples; returns (offsets, ids, dist, keys)."""
    keep, structs = [], []
    for p in parts:
        off = np.ascontiguousarray(p[0], np.int64)
        ids = np.ascontiguousarray(p[1], np.int64)
        dist = np.ascontiguousarray(p[2], np.float32)
        keys = np.ascontiguousarray(p[3], np.float64) if len(p) > 3 and p[3] is not None else None
        keep.append((off, ids, dist, keys))
        structs.append(_c_result(off, ids, dist, keys))
    arr = (ctypes.POINTER(_Result) * len(structs))(*[ctypes.pointer(x) for x in structs])
    base = np.ascontiguousarray(id_base, np.int64)
    out = _Result()
    if k is not None:
        nq = int(len(keep[0][0]) - 1)
        kk = np.ascontiguousarray(np.broadcast_to(np.asarray(k, np.int32), (nq,)), np.int32)
        _check(lib().gts_merge_knn(arr, _ptr(base), len(structs), _ptr(kk), ctypes.byref(out)))
    else:
        _check(lib().gts_merge_range(arr, _ptr(base), len(structs), ctypes.byref(out)))
    res = _host_arrays(out)
    lib().gts_result_free(ctypes.byref(out))
    return res


def merge_knn(parts, id_base, k):
    """kNN answers of shards over disjoint object sets -> the first k by
    (FP64 key, global id); parts carry keys (Index.knn(..., keys=True))."""
    return _merge(parts, id_base, k)


def merge_range(parts, id_base):
    """Range answers of shards -> all answers in ascending global id."""
    return _merge(parts, id_base)


class ShardedIndex:
    """One GTS index per contiguous slice of the objects (shards over disjoint
    object sets, object i of shard s is global id base[s] + i), every query
    sent to every shard, the answers merged exactly (gts_merge_*)."""

    def __init__(self, shards, bases):
        self.shards, self.bases = shards, np.asarray(bases, np.int64)

    @classmethod
    def build(cls, objects, metric: str, n_shards: int, **kw) -> "ShardedIndex":
        n = int(objects.shape[0])
        cuts = [n * s // n_shards for s in range(n_shards + 1)]
        return cls([Index.build(objects[cuts[s]:cuts[s + 1]], metric, **kw) for s in range(n_shards)], cuts[:-1])

    def knn(self, queries, k, **kw) -> Result:
        parts = []
        for ix in self.shards:
            r = ix.knn(queries, k, keys=True, **kw)
            parts.append((r.offsets, r.ids, r.dist, r.keys))
        off, ids, dist, keys = merge_knn(parts, self.bases, k)
        return Result(off, ids, dist, keys=keys)

    def range(self, queries, radii, **kw) -> Result:
        parts = []
        for ix in self.shards:
            r = ix.range(queries, radii, **kw)
            parts.append((r.offsets, r.ids, r.dist))
        off, ids, dist, _ = merge_range(parts, self.bases)
        return Result(off, ids, dist)

    def close(self):
        for ix in self.shards:
            ix.close()


def _multi(fn, columns, queries, per_query, precision, memory_budget):
    if len(columns) != len(queries):
        raise ValueError("one query set per column")
    ms = [_Marshal(q if _is_torch(q) else np.ascontiguousarray(q, np.float32)) for q in queries]
    objs = (_Objects * len(ms))(*[m.obj for m in ms])
    hs = (ctypes.c_void_p * len(columns))(*[c._h.value for c in columns])
    stats = np.zeros(len(STAT_NAMES), np.int64)
    opts = _QueryOpts(precision=PREC_BF16 if precision in ("bf16", PREC_BF16) else PREC_FP32,
                      memory_budget=int(memory_budget), stats=_ptr(stats).value)
    res = _Result()
    _check(fn(hs, len(columns), objs, _ptr(per_query), ctypes.byref(opts), ctypes.byref(res)))
    offsets, ids, dist, kk = _host_arrays(res)
    lib().gts_result_free(ctypes.byref(res))
    return Result(offsets, ids, dist, dict(zip(STAT_NAMES, stats.tolist())), keys=kk)


def multi_range(columns, queries, radii, precision="fp32", memory_budget=0) -> Result:
    """Multi-column range query (gts_multi_range): ``columns`` are indexes
    over the same ids, ``queries`` one [nq, dim_j] array per column (numpy,
    or torch tensors with ``radii`` on the same device); an answer's distance
    is the sum of its column distances (``keys``: the FP64 sums)."""
    r = radii.contiguous() if _is_torch(radii) else np.ascontiguousarray(radii, np.float32)
    return _multi(lib().gts_multi_range, columns, queries, r, precision, memory_budget)


def multi_knn(columns, queries, k, precision="fp32", memory_budget=0) -> Result:
    """Multi-column kNN query (gts_multi_knn), answers in ascending (sum, id)."""
    if _is_torch(k):
        kk = k.contiguous()
    else:
        n = int(queries[0].shape[0])
        kk = np.ascontiguousarray(np.broadcast_to(np.asarray(k, np.int32), (n,)), np.int32)
    return _multi(lib().gts_multi_knn, columns, queries, kk, precision, memory_budget)


def cost_model(n: int, nq: int, p: float, fanout: int, h: int, concurrency: float) -> float:
    """The cost model of Section 5.3 (gts_cost_model)."""
    return float(lib().gts_cost_model(int(n), int(nq), float(p), int(fanout), int(h), float(concurrency)))


def selftest_tc(A, B, a_tmem=False):
    """Diagnostic: D = bf16(A) @ bf16(B).T computed by the tensor-core tile
    primitives (A: [128, K], B: [N, K] float32; a_tmem: A read from TMEM)."""
    A = np.ascontiguousarray(A, np.float32)
    B = np.ascontiguousarray(B, np.float32)
    D = np.zeros((A.shape[0], B.shape[0]), np.float32)
    _check(lib().gts_selftest_tc(_ptr(A), _ptr(B), B.shape[0], A.shape[1], 1 if a_tmem else 0, _ptr(D)))
    return D


def _check(status: int):
    if status != 0:
        L = lib()
        raise GTSError(status, L.gts_status_name(status).decode(), L.gts_last_error().decode())


def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _ptr(x):
    if x is None:
        return None
    if _is_torch(x):
        return ctypes.c_void_p(x.data_ptr())
    return x.ctypes.data_as(ctypes.c_void_p)


def _stream_of(*xs):
    for x in xs:
        if x is not None and _is_torch(x) and x.is_cuda:
            import torch
            return ctypes.c_void_p(torch.cuda.current_stream(x.device).cuda_stream)
    return None


class _Marshal:
    """Keeps the arrays behind a gts_objects alive for the call."""

    def __init__(self, objs):
        self.keep = []
        o = _Objects()
        if isinstance(objs, tuple) or hasattr(objs, "offsets"):
            data, offs = (objs.data, objs.offsets) if hasattr(objs, "offsets") else objs
            if _is_torch(data):
                o.on_device = 1 if data.is_cuda else 0
                data = data.contiguous()
                offs = offs.contiguous()
            else:
                data = np.ascontiguousarray(data, np.uint8)
                offs = np.ascontiguousarray(offs, np.int64)
                if data.size == 0:
                    data = np.zeros(1, np.uint8)
            o.n = int(offs.shape[0]) - 1
            o.dim = 0
            o.data = _ptr(data).value
            o.offsets = _ptr(offs).value
            self.keep += [data, offs]
            self.first = data
        else:
            X = objs
            if _is_torch(X):
                o.on_device = 1 if X.is_cuda else 0
                X = X.contiguous()
            else:
                X = np.ascontiguousarray(X, np.float32)
            if X.ndim != 2:
                raise ValueError("vectors must be 2-D [n, dim]")
            o.n = int(X.shape[0])
            o.dim = int(X.shape[1])
            count = X.numel() if _is_torch(X) else X.size
            o.data = _ptr(X).value if count else None
            self.keep.append(X)
            self.first = X
        self.obj = o


class Result:
    """CSR answers: ids/dist[offsets[i]:offsets[i+1]] belong to query i
    (``keys``: the answers' FP64 keys, kNN with ``keys=True``)."""

    def __init__(self, offsets, ids, dist, stats=None, device_result=None, keys=None):
        self.offsets, self.ids, self.dist, self.stats = offsets, ids, dist, stats
        self.keys = keys
        self._dev = device_result

    def query(self, i):
        a, b = int(self.offsets[i]), int(self.offsets[i + 1])
        return self.ids[a:b], self.dist[a:b]

    def copy_to(self, offsets, ids, dist):
        """Copy a device-resident result into caller arrays (numpy or torch,
        host or device)."""
        _check(lib().gts_result_copy(ctypes.byref(self._dev), _ptr(offsets), _ptr(ids), _ptr(dist)))

    def free(self):
        if self._dev is not None:
            lib().gts_result_free(ctypes.byref(self._dev))
            self._dev = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class Index:
    """A GTS index held on the current CUDA device (owned by the library)."""

    def __init__(self, handle, metric: str):
        self._h = handle
        self.metric = metric

    @classmethod
    def build(cls, objects, metric: str, n_pivots: int = 0, fanout: int = 20, root_pivot: int = -1,
              seed: int = 0, cache_limit: int = 0, stream=None) -> "Index":
        m = _Marshal(objects)
        opts = _BuildOpts(stream=stream if stream is not None else _stream_of(m.first), root_pivot=int(root_pivot),
                          seed=int(seed), cache_limit=int(cache_limit))
        h = ctypes.c_void_p()
        _check(lib().gts_build(ctypes.byref(m.obj), METRIC_IDS[metric], int(n_pivots), int(fanout),
                               ctypes.byref(opts), ctypes.byref(h)))
        return cls(h, metric)

    def _query(self, fn, queries, per_query, precision, result_on_device, memory_budget, seq, stream, timing=False,
               count_table_pass=False, keys=False):
        m = _Marshal(queries)
        stats = np.zeros(len(STAT_NAMES), np.int64)
        stage = np.zeros(2 * len(STAGE_NAMES), np.float64) if timing else None
        opts = _QueryOpts(stream=stream if stream is not None else _stream_of(m.first),
                          precision=PREC_BF16 if precision in ("bf16", PREC_BF16) else PREC_FP32,
                          result_on_device=1 if result_on_device else 0, memory_budget=int(memory_budget),
                          seq=_ptr(seq).value if seq is not None else None, stats=_ptr(stats).value,
                          stage_ms=_ptr(stage).value if timing else None,
                          flags=(QUERY_COUNT_TABLE_PASS if count_table_pass else 0) | (QUERY_KEYS if keys else 0))
        res = _Result()
        _check(fn(self._h, ctypes.byref(m.obj), _ptr(per_query), ctypes.byref(opts), ctypes.byref(res)))
        st = dict(zip(STAT_NAMES, stats.tolist()))
        if timing:
            k = len(STAGE_NAMES)
            st["stage_ms"] = dict(zip(STAGE_NAMES, stage[:k].tolist()))
            st["stage_launches"] = dict(zip(STAGE_NAMES, stage[k:].astype(int).tolist()))
        nq = int(res.nq)
        if res.on_device:
            return Result(res.offsets, res.ids, res.dist, st, device_result=res)
        offsets, ids, dist, kk = _host_arrays(res)
        lib().gts_result_free(ctypes.byref(res))
        return Result(offsets, ids, dist, st, keys=kk)

    def range(self, queries, radii, precision="fp32", result_on_device=False, memory_budget=0, seq=None,
              stream=None, timing=False, count_table_pass=False) -> Result:
        if _is_torch(radii):
            r = radii.contiguous()
        else:
            r = np.ascontiguousarray(radii, np.float32)
        return self._query(lib().gts_range, queries, r, precision, result_on_device, memory_budget, seq, stream,
                           timing, count_table_pass)

    def knn(self, queries, k, precision="fp32", result_on_device=False, memory_budget=0, seq=None,
            stream=None, timing=False, count_table_pass=False, keys=False) -> Result:
        if _is_torch(k):
            kk = k.contiguous()
        else:
            n = queries.shape[0] if hasattr(queries, "shape") else (
                queries.n if hasattr(queries, "n") else int(queries[1].shape[0]) - 1)
            kk = np.ascontiguousarray(np.broadcast_to(np.asarray(k, np.int32), (n,)), np.int32)
        return self._query(lib().gts_knn, queries, kk, precision, result_on_device, memory_budget, seq, stream,
                           timing, count_table_pass, keys)

    def save(self, path: str):
        """Write the whole index to a file (gts_save)."""
        _check(lib().gts_save(self._h, os.fsencode(path)))

    @classmethod
    def load(cls, path: str, metric: Optional[str] = None, stream=None, cache_limit: int = 0) -> "Index":
        """Read an index written by save onto the current device (gts_load)."""
        opts = _BuildOpts(stream=stream, root_pivot=-1, seed=0, cache_limit=int(cache_limit))
        h = ctypes.c_void_p()
        _check(lib().gts_load(os.fsencode(path), ctypes.byref(opts), ctypes.byref(h)))
        ix = cls(h, metric or "")
        ix.metric = {EDIT: "edit", L1: "l1", L2: "l2", COS: "cos"}[ix.info()["metric"]]
        return ix

    def get_tuning(self) -> dict:
        t = _Tuning()
        _check(lib().gts_get_tuning(self._h, ctypes.byref(t)))
        return {f: int(getattr(t, f)) for f in TUNING_FIELDS + ["tuned"]}

    def set_tuning(self, **kw):
        cur = self.get_tuning()
        cur.update(kw)
        t = _Tuning(**{f: int(cur[f]) for f in TUNING_FIELDS})
        _check(lib().gts_set_tuning(self._h, ctypes.byref(t)))

    def autotune(self, queries, k=None, radii=None, precision="fp32", reps=3, memory_budget=0, stream=None) -> dict:
        """Time the sample batch under each candidate setting and keep the
        fastest (gts_autotune); returns the chosen setting."""
        m = _Marshal(queries)
        n = m.obj.n
        kk = None if k is None else np.ascontiguousarray(np.broadcast_to(np.asarray(k, np.int32), (n,)), np.int32)
        rr = None if radii is None else np.ascontiguousarray(np.broadcast_to(np.asarray(radii, np.float32), (n,)),
                                                             np.float32)
        if m.obj.on_device:
            import torch
            kk = None if kk is None else torch.from_numpy(kk.copy()).cuda()
            rr = None if rr is None else torch.from_numpy(rr.copy()).cuda()
        opts = _QueryOpts(stream=stream if stream is not None else _stream_of(m.first),
                          precision=PREC_BF16 if precision in ("bf16", PREC_BF16) else PREC_FP32,
                          memory_budget=int(memory_budget))
        out = _Tuning()
        _check(lib().gts_autotune(self._h, ctypes.byref(m.obj), _ptr(rr) if rr is not None else None,
                                  _ptr(kk) if kk is not None else None, ctypes.byref(opts), int(reps),
                                  ctypes.byref(out)))
        return {f: int(getattr(out, f)) for f in TUNING_FIELDS + ["tuned"]}

    def autotune_shape(self, queries, k=None, radii=None, precision="fp32", candidates=4, reps=2,
                       memory_budget=0, stream=None) -> list:
        """Rank index shapes (fanout, pivot levels) by the cost model of
        Section 5.3, rebuild and time the cheapest ones on the sample batch and
        keep the fastest (gts_autotune_shape); returns the shapes timed,
        fastest first."""
        m = _Marshal(queries)
        n = m.obj.n
        kk = None if k is None else np.ascontiguousarray(np.broadcast_to(np.asarray(k, np.int32), (n,)), np.int32)
        rr = None if radii is None else np.ascontiguousarray(np.broadcast_to(np.asarray(radii, np.float32), (n,)),
                                                             np.float32)
        if m.obj.on_device:
            import torch
            kk = None if kk is None else torch.from_numpy(kk.copy()).cuda()
            rr = None if rr is None else torch.from_numpy(rr.copy()).cuda()
        opts = _QueryOpts(stream=stream if stream is not None else _stream_of(m.first),
                          precision=PREC_BF16 if precision in ("bf16", PREC_BF16) else PREC_FP32,
                          memory_budget=int(memory_budget))
        out = (_Shape * (int(candidates) + 1))()
        cnt = ctypes.c_int32()
        _check(lib().gts_autotune_shape(self._h, ctypes.byref(m.obj), _ptr(rr) if rr is not None else None,
                                        _ptr(kk) if kk is not None else None, ctypes.byref(opts), int(candidates),
                                        int(reps), out, ctypes.byref(cnt)))
        return [dict(fanout=out[i].fanout, n_pivots=out[i].n_pivots, model_cost=out[i].model_cost,
                     measured_ms=out[i].measured_ms) for i in range(cnt.value)]

    def insert(self, objects) -> np.ndarray:
        m = _Marshal(objects)
        ids = np.zeros(max(1, m.obj.n), np.int64)
        _check(lib().gts_insert(self._h, ctypes.byref(m.obj), _ptr(ids)))
        return ids[:m.obj.n]

    def delete(self, ids) -> int:
        ids = np.ascontiguousarray(ids, np.int64)
        missing = np.zeros(1, np.int64)
        st = lib().gts_delete(self._h, _ptr(ids) if ids.size else None, int(ids.size), _ptr(missing))
        if st not in (0, 5):
            _check(st)
        return int(missing[0])

    def batch_update(self, objects=None, delete_ids=None) -> np.ndarray:
        m = _Marshal(objects) if objects is not None else None
        d = np.ascontiguousarray(delete_ids if delete_ids is not None else np.zeros(0), np.int64)
        ids = np.zeros(max(1, m.obj.n if m else 0), np.int64)
        st = lib().gts_batch_update(self._h, ctypes.byref(m.obj) if m else None, _ptr(d) if d.size else None,
                                    int(d.size), _ptr(ids))
        if st not in (0, 5):
            _check(st)
        return ids[:(m.obj.n if m else 0)]

    def rebuild(self):
        _check(lib().gts_rebuild(self._h))

    def info(self) -> dict:
        i = _Info()
        _check(lib().gts_info(self._h, ctypes.byref(i)))
        return {f: getattr(i, f) for f, _ in _Info._fields_}

    def tree_level(self, level: int) -> dict:
        F = self.info()["fanout"]
        cnt = F ** level
        out = dict(pos=np.zeros(cnt, np.int64), size=np.zeros(cnt, np.int64), lo=np.zeros(cnt, np.float32),
                   hi=np.zeros(cnt, np.float32), pivot=np.zeros(cnt, np.int64))
        _check(lib().gts_tree_level(self._h, int(level), _ptr(out["pos"]), _ptr(out["size"]), _ptr(out["lo"]),
                                    _ptr(out["hi"]), _ptr(out["pivot"])))
        return out

    def table(self):
        inf = self.info()
        n, h = inf["n_tree"], inf["h"]
        ids = np.zeros(max(n, 1), np.int64)
        tab = np.zeros(max(h * n, 1), np.float32)
        _check(lib().gts_table(self._h, _ptr(ids), _ptr(tab)))
        return ids[:n], tab[:h * n].reshape(h, n)

    def close(self):
        if self._h:
            lib().gts_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching request loop over an index (gts_serve_*)."""

    def __init__(self, index: "Index", max_batch=0, n_streams=0, precision="fp32", result_budget=0,
                 memory_budget=0, batch_quantum=0):
        o = _ServeOpts(max_batch=int(max_batch), n_streams=int(n_streams),
                       precision=PREC_BF16 if precision in ("bf16", PREC_BF16) else PREC_FP32,
                       batch_quantum=int(batch_quantum), result_budget=int(result_budget),
                       memory_budget=int(memory_budget))
        self._h = ctypes.c_void_p()
        self.index = index
        _check(lib().gts_serve_start(index._h, ctypes.byref(o), ctypes.byref(self._h)))

    def submit(self, query, kind: str, param) -> int:
        """kind 'range' (param = radius) or 'knn' (param = k); returns a ticket."""
        if isinstance(query, (bytes, bytearray)):
            buf = np.frombuffer(bytes(query) or b"\0", np.uint8)
            n = len(query)
        else:
            buf = np.ascontiguousarray(query, np.float32)
            n = buf.size
        t = ctypes.c_int64()
        _check(lib().gts_serve_submit(self._h, _ptr(buf), n, 0 if kind == "range" else 1, float(param),
                                      ctypes.byref(t)))
        return int(t.value)

    def wait(self, ticket: int, timeout_ms: int = -1):
        """(ids, dist, latency_ms) of a request."""
        res = _Result()
        lat = ctypes.c_double()
        _check(lib().gts_serve_wait(self._h, int(ticket), int(timeout_ms), ctypes.byref(res), ctypes.byref(lat)))
        m = int(np.ctypeslib.as_array(ctypes.cast(res.offsets, ctypes.POINTER(ctypes.c_int64)), (2,))[1])
        ids = np.ctypeslib.as_array(ctypes.cast(res.ids, ctypes.POINTER(ctypes.c_int64)), (max(m, 1),))[:m].copy()
        dist = np.ctypeslib.as_array(ctypes.cast(res.dist, ctypes.POINTER(ctypes.c_float)), (max(m, 1),))[:m].copy()
        lib().gts_result_free(ctypes.byref(res))
        return ids, dist, float(lat.value)

    def stats(self) -> dict:
        out = np.zeros(6, np.int64)
        _check(lib().gts_serve_stats(self._h, _ptr(out), 6))
        return dict(batches=int(out[0]), requests=int(out[1]), max_batch=int(out[2]), max_in_flight=int(out[3]),
                    projected_bytes=int(out[4]), below_worst_case=int(out[5]))

    def project(self, query, kind: str, param) -> int:
        """The admission projection (bytes) of one request, not submitted."""
        if isinstance(query, (bytes, bytearray)):
            buf = np.frombuffer(bytes(query) or b"\0", np.uint8)
            n = len(query)
        else:
            buf = np.ascontiguousarray(query, np.float32)
            n = buf.size
        out = np.zeros(1, np.int64)
        _check(lib().gts_serve_project(self._h, _ptr(buf), n, 0 if kind == "range" else 1, float(param), _ptr(out)))
        return int(out[0])

    def stop(self):
        if self._h:
            _check(lib().gts_serve_stop(self._h))
            self._h = None
