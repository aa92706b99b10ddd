"""CPU oracle (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package. It wraps ``oracle.c`` (plain C, FP64),
compiled in place, through ctypes:

* ``exact_knn``  - O1, Definition 1 of the paper (exact range-filtered k-NN);
* ``search``     - O2, the literal HSIG search (Strategies A, B, C and the
                   range-aware selection of Section 4.2);
* ``route``      - range bounds, segment masks and strategies by definition.

See the header of ``oracle.c`` for the readings of the paper it follows.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

STRATEGY = {"pre": 0, "hybrid": 1, "post": 2, "auto": -1}
P = ctypes.c_void_p


def compile(force: bool = False) -> str:
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", _SRC,
           "-o", _LIB + ".tmp", "-lpthread", "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(_LIB + ".tmp", _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            compile()
            lib = ctypes.CDLL(_LIB)
            lib.orc_index_open.argtypes = [ctypes.c_char_p, ctypes.POINTER(P)]
            lib.orc_index_open.restype = ctypes.c_int
            lib.orc_index_close.argtypes = [P]
            lib.orc_index_close.restype = None
            lib.orc_index_max_level.argtypes = [P]
            lib.orc_index_max_level.restype = ctypes.c_int
            lib.orc_exact_knn_batch.argtypes = [P, P, ctypes.c_int64, ctypes.c_int, P, P, P,
                                                ctypes.c_int64, ctypes.c_int, ctypes.c_int, P, P, P]
            lib.orc_exact_knn_batch.restype = ctypes.c_int
            lib.orc_search_batch.argtypes = [P, P, P, P, ctypes.c_int64, ctypes.c_int, ctypes.c_int,
                                             ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int64,
                                             ctypes.c_int64, ctypes.c_int, P, P, P, P, P, P]
            lib.orc_search_batch.restype = ctypes.c_int
            lib.orc_search_batch_sel.argtypes = lib.orc_search_batch.argtypes + [ctypes.c_int]
            lib.orc_search_batch_sel.restype = ctypes.c_int
            lib.orc_search_batch_ex.argtypes = lib.orc_search_batch_sel.argtypes + [P, P, P]
            lib.orc_search_batch_ex.restype = ctypes.c_int
            lib.orc_search_batch_tr.argtypes = lib.orc_search_batch_ex.argtypes + [P]
            lib.orc_search_batch_tr.restype = ctypes.c_int
            lib.orc_exact_knn_batch2.argtypes = [P, P, P, ctypes.c_int64, ctypes.c_int, P, P, P, P, P,
                                                 ctypes.c_int64, ctypes.c_int, ctypes.c_int, P, P, P]
            lib.orc_exact_knn_batch2.restype = ctypes.c_int
            lib.orc_route_batch.argtypes = [P, P, P, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                            P, P, P, P, P]
            lib.orc_route_batch.restype = ctypes.c_int
            lib.orc_segment_mask.argtypes = [P, ctypes.c_int64, ctypes.c_int64]
            lib.orc_segment_mask.restype = ctypes.c_uint32
            lib.orc_skiplist_first.argtypes = [P, ctypes.c_int64]
            lib.orc_skiplist_first.restype = ctypes.c_int32
            _lib = lib
    return _lib


def _p(a):
    return a.ctypes.data if a is not None else None


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


def default_threads() -> int:
    return max(1, len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count() or 1)


def exact_knn(vectors, attrs, queries, lo, hi, k, threads=None, attr2=None, lo2=None, hi2=None):
    """O1. Returns (ids int64 [nq,k], dist float64 [nq,k], count int64 [nq]). With
    attr2 (one value per object) the range is lo <= attr <= hi AND lo2 <= attr2 <= hi2."""
    lib = _load()
    X, A = _c(vectors, np.float32), _c(attrs, np.int64)
    Q = _c(queries, np.float32).reshape(-1, X.shape[1])
    lo, hi = _c(lo, np.int64), _c(hi, np.int64)
    nq = Q.shape[0]
    ids = np.empty((nq, k), np.int64)
    dist = np.empty((nq, k), np.float64)
    cnt = np.empty(nq, np.int64)
    A2 = _c(attr2, np.int64) if attr2 is not None else None
    lo2 = _c(lo2, np.int64) if attr2 is not None else None
    hi2 = _c(hi2, np.int64) if attr2 is not None else None
    rc = lib.orc_exact_knn_batch2(_p(X), _p(A), _p(A2), X.shape[0], X.shape[1], _p(Q), _p(lo), _p(hi),
                                  _p(lo2), _p(hi2), nq, k, threads or default_threads(), _p(ids), _p(dist),
                                  _p(cnt))
    if rc != 0:
        raise RuntimeError(f"orc_exact_knn_batch failed: {rc}")
    return ids, dist, cnt


class OracleIndex:
    """An index file opened by the oracle's own reader (checksums verified)."""

    def __init__(self, path: str):
        self._lib = _load()
        h = P()
        rc = self._lib.orc_index_open(path.encode(), ctypes.byref(h))
        if rc != 0:
            raise RuntimeError(f"oracle could not open {path}: code {rc}")
        self._h = h
        self.path = path
        self.max_level = int(self._lib.orc_index_max_level(h))

    def close(self):
        if getattr(self, "_h", None):
            self._lib.orc_index_close(self._h)
            self._h = None

    def __del__(self):
        self.close()

    def search(self, queries, lo, hi, k, ef=100, m=16, ef_post=None, strategy="auto",
               tau_a=0, tau_b=0, threads=None, selection=2, attr2=None, lo2=None, hi2=None, trace=False):
        """O2. Returns dict(ids, dist, count, strategy, n_dist, n_exp). selection: 2 = S2
        (first ceil(m/S') slots per intersected chunk), 1 = S1 (the m neighbours nearest
        to the expanded object over all intersected chunks). attr2/lo2/hi2 add the
        conjunctive predicate lo2 <= attr2 <= hi2 on a second attribute (R9). With
        ``trace`` the dict also holds ``eps`` [nq, max_level + 1]: the entry point each
        layer l of the hierarchical descent started from (column l; -1 where no layer
        was searched)."""
        Q = _c(queries, np.float32)
        lo, hi = _c(lo, np.int64), _c(hi, np.int64)
        nq = lo.shape[0]
        out = dict(ids=np.empty((nq, k), np.int64), dist=np.empty((nq, k), np.float64),
                   count=np.empty(nq, np.int64), strategy=np.empty(nq, np.int32),
                   n_dist=np.empty(nq, np.int64), n_exp=np.empty(nq, np.int64))
        st = STRATEGY[strategy] if isinstance(strategy, str) else int(strategy)
        A2 = _c(attr2, np.int64) if attr2 is not None else None
        l2 = _c(lo2, np.int64) if attr2 is not None else None
        h2 = _c(hi2, np.int64) if attr2 is not None else None
        eps = np.empty((nq, self.max_level + 1), np.int32) if trace else None
        rc = self._lib.orc_search_batch_tr(self._h, _p(Q), _p(lo), _p(hi), nq, k, ef, m, ef_post or ef, st,
                                           tau_a, tau_b, threads or default_threads(), _p(out["ids"]),
                                           _p(out["dist"]), _p(out["count"]), _p(out["strategy"]),
                                           _p(out["n_dist"]), _p(out["n_exp"]), int(selection),
                                           _p(A2), _p(l2), _p(h2), _p(eps))
        if trace:
            out["eps"] = eps
        if rc != 0:
            raise RuntimeError(f"orc_search_batch failed: {rc}")
        return out

    def route(self, lo, hi, tau_a=0, tau_b=0):
        """Range bounds, masks and strategies by definition, plus skip-list descent."""
        lo, hi = _c(lo, np.int64), _c(hi, np.int64)
        nq = lo.shape[0]
        out = dict(pa=np.empty(nq, np.int64), pb=np.empty(nq, np.int64), mask=np.empty(nq, np.uint32),
                   strategy=np.empty(nq, np.int32), first=np.empty(nq, np.int32))
        rc = self._lib.orc_route_batch(self._h, _p(lo), _p(hi), nq, tau_a, tau_b, _p(out["pa"]),
                                       _p(out["pb"]), _p(out["mask"]), _p(out["strategy"]), _p(out["first"]))
        if rc != 0:
            raise RuntimeError(f"orc_route_batch failed: {rc}")
        return out


def recall(found_ids, exact_ids, exact_count, k):
    """Eq. 1: |kNN' ∩ kNN| / min(k, |R|); a query with |R| = 0 scores 1."""
    found_ids = np.asarray(found_ids)
    exact_ids = np.asarray(exact_ids)
    out = np.empty(found_ids.shape[0], np.float64)
    for i in range(found_ids.shape[0]):
        c = int(min(k, exact_count[i]))
        if c == 0:
            out[i] = 1.0
            continue
        ex = set(int(v) for v in exact_ids[i, :c])
        fo = set(int(v) for v in found_ids[i, :k] if v >= 0)
        out[i] = len(ex & fo) / c
    return out
