"""GB300 range-filtered k-NN search over an HSIG (UNIFY, Section 4.2).

Thin ctypes binding of ``libunify.so`` (the C ABI in ``include/unify.h``).
Every step of the search runs in the library's CUDA kernels; PyTorch is used
only to own device memory and streams. The binding refuses to work when the
compiled library is missing: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading
import weakref

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libunify.so")

PRE, HYBRID, POST, AUTO = 0, 1, 2, -1
STRATEGIES = {"pre": PRE, "hybrid": HYBRID, "post": POST, "auto": AUTO}
FP32, BF16, FP8E4M3 = 0, 1, 2
Q_LIMIT, Q_TRUNCATED = 1, 2

_P = ctypes.c_void_p
_lock = threading.Lock()
_lib = None


class UnifyError(RuntimeError):
    pass


class Params(ctypes.Structure):
    """Mirror of unify_params_t."""
    _fields_ = [("ef", ctypes.c_int), ("m", ctypes.c_int), ("ef_post", ctypes.c_int),
                ("rerank_mult", ctypes.c_int), ("dtype", ctypes.c_int), ("tau_a", ctypes.c_int64),
                ("tau_b", ctypes.c_int64), ("cand_cap", ctypes.c_int), ("visited_cap", ctypes.c_int),
                ("max_expansions", ctypes.c_int), ("warps_per_block", ctypes.c_int),
                ("scan_rows", ctypes.c_int), ("reg_budget", ctypes.c_int), ("tc_scan", ctypes.c_int), ("selection", ctypes.c_int)]

    @classmethod
    def defaults(cls, **kw) -> "Params":
        p = cls()
        lib().unify_default_params(ctypes.byref(p))
        for k, v in kw.items():
            if not hasattr(p, k):
                raise KeyError(k)
            setattr(p, k, v)
        return p


def build(force: bool = False) -> str:
    from . import buildlib as _b
    return _b.build(force=force)


def lib():
    """The loaded CUDA library; raises when it was not built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise UnifyError(f"CUDA library not built: {LIB_PATH} is missing (run build())")
            L = ctypes.CDLL(LIB_PATH)
            L.unify_default_params.argtypes = [_P]
            L.unify_default_params.restype = None
            L.unify_load_index.argtypes = [ctypes.c_char_p, ctypes.c_int, ctypes.POINTER(_P)]
            L.unify_load_index.restype = ctypes.c_int
            L.unify_free_index.argtypes = [_P]
            L.unify_free_index.restype = None
            L.unify_index_info.argtypes = [_P, _P, _P, _P, _P, _P]
            L.unify_index_info.restype = ctypes.c_int
            L.unify_route.argtypes = [_P, _P, _P, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                      _P, _P, _P, _P, _P]
            L.unify_route.restype = ctypes.c_int
            L.unify_search.argtypes = [_P, _P, _P, _P, ctypes.c_int64, ctypes.c_int, ctypes.c_int,
                                       ctypes.c_int, _P, _P, _P, _P, _P, _P, _P]
            L.unify_search.restype = ctypes.c_int
            L.unify_search_conj.argtypes = [_P, _P, _P, _P, _P, _P, _P, ctypes.c_int64, ctypes.c_int, ctypes.c_int,
                                            ctypes.c_int, _P, _P, _P, _P, _P, _P, _P]
            L.unify_search_conj.restype = ctypes.c_int
            L.unify_search_auto.argtypes = [_P, _P, _P, _P, ctypes.c_int64, ctypes.c_int, ctypes.c_int,
                                            _P, _P, _P, _P, _P, _P]
            L.unify_search_auto.restype = ctypes.c_int
            L.unify_search_auto_host.argtypes = [_P, _P, _P, _P, ctypes.c_int64, ctypes.c_int,
                                                 ctypes.c_int, _P, _P, _P, _P, _P, _P]
            L.unify_search_auto_host.restype = ctypes.c_int
            L.unify_plan_create.argtypes = [_P, _P, _P, _P, ctypes.c_int64, ctypes.c_int, ctypes.c_int,
                                            ctypes.c_int, _P, _P, _P, _P, _P, ctypes.POINTER(_P)]
            L.unify_plan_create.restype = ctypes.c_int
            L.unify_plan_launch.argtypes = [_P, _P]
            L.unify_plan_launch.restype = ctypes.c_int
            L.unify_plan_destroy.argtypes = [_P]
            L.unify_plan_destroy.restype = None
            L.unify_timing_enable.argtypes = [_P, ctypes.c_int]
            L.unify_timing_enable.restype = ctypes.c_int
            L.unify_timing_collect.argtypes = [_P, _P, _P]
            L.unify_timing_collect.restype = ctypes.c_int
            L.unify_last_error.argtypes = []
            L.unify_last_error.restype = ctypes.c_char_p
            L.unify_build_assist_create.argtypes = [ctypes.c_int, _P]
            L.unify_build_assist_create.restype = ctypes.c_int
            L.unify_build_assist_destroy.argtypes = [_P]
            L.unify_build_assist_destroy.restype = None
            _lib = L
    return _lib


def _check(rc: int, what: str):
    if rc != 0:
        raise UnifyError(f"{what} failed ({rc}): {lib().unify_last_error().decode()}")


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream_handle(torch, device):
    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


class Index:
    """An HSIG index resident on one GPU."""

    def __init__(self, path: str, device: int = 0):
        import torch
        self._torch = torch
        self.device = torch.device("cuda", device)
        h = _P()
        _check(lib().unify_load_index(path.encode(), device, ctypes.byref(h)), "unify_load_index")
        self._h = h
        n, d, S, M, L = ctypes.c_int64(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(lib().unify_index_info(h, ctypes.byref(n), ctypes.byref(d), ctypes.byref(S), ctypes.byref(M),
                                      ctypes.byref(L)), "unify_index_info")
        self.n, self.d, self.S, self.M, self.max_level = n.value, d.value, S.value, M.value, L.value
        self._plans = weakref.WeakSet()

    def close(self):
        for p in list(getattr(self, "_plans", ())):
            p.close()
        if getattr(self, "_h", None):
            lib().unify_free_index(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- helpers
    def _dev(self, x, dtype):
        t = self._torch.as_tensor(x)
        return t.to(device=self.device, dtype=dtype).contiguous()

    def route(self, lo, hi, tau_a: int = -1, tau_b: int = -1):
        torch = self._torch
        lo, hi = self._dev(lo, torch.int64), self._dev(hi, torch.int64)
        nq = lo.numel()
        out = {k: torch.empty(nq, dtype=torch.int32, device=self.device) for k in ("pa", "pb", "mask", "strategy")}
        _check(lib().unify_route(self._h, _ptr(lo), _ptr(hi), nq, tau_a, tau_b, _ptr(out["pa"]), _ptr(out["pb"]),
                                 _ptr(out["mask"]), _ptr(out["strategy"]), _stream_handle(torch, self.device)),
               "unify_route")
        return out

    def search(self, q, lo, hi, k: int, ef: int = 0, strategy="auto", params: Params | None = None,
               out=None, counters: bool = False, attr2=None, lo2=None, hi2=None):
        """Returns dict(ids int64 [nq,k], dist float32 [nq,k], count int32 [nq], status int32 [nq]
        [, counters int32 [nq,4]: distance evaluations, expansions, start and end in microseconds])
        as device tensors. ``out`` may pass preallocated tensors. With ``attr2`` (one value per
        object) and ``lo2``/``hi2`` (one range per query) the search is conjunctive
        (unify_search_conj)."""
        torch = self._torch
        q = self._dev(q, torch.float32).reshape(-1, self.d)
        lo, hi = self._dev(lo, torch.int64), self._dev(hi, torch.int64)
        nq = q.shape[0]
        if lo.numel() != nq or hi.numel() != nq:
            raise ValueError("q, lo and hi must have the same number of queries")
        st = STRATEGIES[strategy] if isinstance(strategy, str) else int(strategy)
        if out is None:
            out = dict(ids=torch.empty((nq, k), dtype=torch.int64, device=self.device),
                       dist=torch.empty((nq, k), dtype=torch.float32, device=self.device),
                       count=torch.empty(nq, dtype=torch.int32, device=self.device),
                       status=torch.empty(nq, dtype=torch.int32, device=self.device))
            if counters:
                out["counters"] = torch.empty((nq, 4), dtype=torch.int32, device=self.device)
        p = ctypes.byref(params) if params is not None else None
        if attr2 is not None:
            a2 = self._dev(attr2, torch.int64)
            l2, h2 = self._dev(lo2, torch.int64), self._dev(hi2, torch.int64)
            if a2.numel() != self.n or l2.numel() != nq or h2.numel() != nq:
                raise ValueError("attr2 needs one value per object, lo2 and hi2 one per query")
            _check(lib().unify_search_conj(self._h, _ptr(q), _ptr(lo), _ptr(hi), _ptr(a2), _ptr(l2), _ptr(h2), nq,
                                           k, ef, st, p, _ptr(out["ids"]), _ptr(out["dist"]), _ptr(out["count"]),
                                           _ptr(out.get("status")), _ptr(out.get("counters")),
                                           _stream_handle(torch, self.device)),
                   "unify_search_conj")
            return out
        _check(lib().unify_search(self._h, _ptr(q), _ptr(lo), _ptr(hi), nq, k, ef, st, p, _ptr(out["ids"]),
                                  _ptr(out["dist"]), _ptr(out["count"]), _ptr(out.get("status")),
                                  _ptr(out.get("counters")), _stream_handle(torch, self.device)),
               "unify_search")
        return out

    PHASES = ("route", "search", "tcscan", "unused3")

    def plan(self, q, lo, hi, k: int, ef: int = 0, strategy="auto", params: Params | None = None):
        """Captures a search of these device buffers into a CUDA graph (see Plan)."""
        p = Plan(self, q, lo, hi, k, ef, strategy, params)
        self._plans.add(p)
        return p

    def timing(self, enable: bool = True):
        _check(lib().unify_timing_enable(self._h, 1 if enable else 0), "unify_timing_enable")

    def collect_timing(self) -> dict:
        """{phase: (summed milliseconds, spans)} of the searches since the last collect."""
        ms = (ctypes.c_double * 4)()
        cnt = (ctypes.c_int64 * 4)()
        _check(lib().unify_timing_collect(self._h, ms, cnt), "unify_timing_collect")
        return {ph: (ms[i], cnt[i]) for i, ph in enumerate(self.PHASES)}

    def search_auto(self, q, lo, hi, k: int, ef: int = 0, params: Params | None = None, out=None):
        return self.search(q, lo, hi, k, ef=ef, strategy=AUTO, params=params, out=out)

    def search_auto_host(self, q: np.ndarray, lo: np.ndarray, hi: np.ndarray, k: int, ef: int = 0,
                         params: Params | None = None, out=None):
        """Host buffers in and out (numpy arrays or pinned CPU tensors); synchronous."""
        q = np.ascontiguousarray(q, dtype=np.float32) if isinstance(q, np.ndarray) else q
        lo = np.ascontiguousarray(lo, dtype=np.int64) if isinstance(lo, np.ndarray) else lo
        hi = np.ascontiguousarray(hi, dtype=np.int64) if isinstance(hi, np.ndarray) else hi
        nq = lo.shape[0]
        if out is None:
            out = dict(ids=np.empty((nq, k), np.int64), dist=np.empty((nq, k), np.float32),
                       count=np.empty(nq, np.int32), status=np.empty(nq, np.uint32))

        def hp(a):
            return ctypes.c_void_p(a.ctypes.data) if isinstance(a, np.ndarray) else ctypes.c_void_p(a.data_ptr())

        p = ctypes.byref(params) if params is not None else None
        _check(lib().unify_search_auto_host(self._h, hp(q), hp(lo), hp(hi), nq, k, ef, p, hp(out["ids"]),
                                            hp(out["dist"]), hp(out["count"]), hp(out["status"]),
                                            _stream_handle(self._torch, self.device)),
               "unify_search_auto_host")
        return out


class Plan:
    """A search captured into a CUDA graph for fixed device buffers. ``launch()``
    replays it on the current stream; update ``q``, ``lo``, ``hi`` in place between
    launches. Results land in ``out`` (ids, dist, count, status)."""

    def __init__(self, index: Index, q, lo, hi, k, ef=0, strategy="auto", params=None):
        torch = index._torch
        self.index = index
        self.q = index._dev(q, torch.float32).reshape(-1, index.d)
        self.lo = index._dev(lo, torch.int64)
        self.hi = index._dev(hi, torch.int64)
        nq = self.q.shape[0]
        self.out = dict(ids=torch.empty((nq, k), dtype=torch.int64, device=index.device),
                        dist=torch.empty((nq, k), dtype=torch.float32, device=index.device),
                        count=torch.empty(nq, dtype=torch.int32, device=index.device),
                        status=torch.empty(nq, dtype=torch.int32, device=index.device))
        st = STRATEGIES[strategy] if isinstance(strategy, str) else int(strategy)
        self._params = params if params is not None else Params.defaults()
        h = _P()
        _check(lib().unify_plan_create(index._h, _ptr(self.q), _ptr(self.lo), _ptr(self.hi), nq, k, ef, st,
                                       ctypes.byref(self._params), _ptr(self.out["ids"]), _ptr(self.out["dist"]),
                                       _ptr(self.out["count"]), _ptr(self.out["status"]), ctypes.byref(h)),
               "unify_plan_create")
        self._h = h

    def launch(self):
        _check(lib().unify_plan_launch(self._h, _stream_handle(self.index._torch, self.index.device)),
               "unify_plan_launch")
        return self.out

    def close(self):
        if getattr(self, "_h", None):
            lib().unify_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def build_index_gpu(vectors: np.ndarray, attrs: np.ndarray, path: str, S: int, M: int, efc: int,
                    seed: int = 0, threads: int = 0, device: int = 0, device_apply: bool = True) -> str:
    """HSIG construction (Algorithms 4-6) with the proposal step of every batch of
    64 or more nodes (descent, ANNSearch and pruning per node and segment) on GPU
    ``device``. With ``device_apply`` the GPU also stores the forward lists and
    applies the reverse edges (Algorithm 4) from the first proposal on, and the graph
    returns to the host once, before the skip list and Algorithm 5; otherwise the host
    applies every batch's edges. Entry points stay on the host, which writes the
    file. Needs M <= 32, efc <= 256, d <= 1024, S <= 32."""
    import hsig_build
    L = lib()
    ctx = _P()
    _check(L.unify_build_assist_create(device, ctypes.byref(ctx)), "unify_build_assist_create")
    try:
        fns = [ctypes.cast(f, _P).value for f in (L.unify_build_propose, L.unify_build_apply, L.unify_build_fetch)]
        if not device_apply:
            fns[1] = fns[2] = None
        try:
            return hsig_build.build_index(vectors, attrs, path, S, M, efc, seed=seed, threads=threads,
                                          assist=(*fns, ctx.value))
        except RuntimeError as e:
            raise UnifyError(f"{e}: {L.unify_last_error().decode()}") from None
    finally:
        L.unify_build_assist_destroy(ctx)


def assisted_build_is_exact(vectors: np.ndarray) -> bool:
    """True when every coordinate is an integer and d * (max - min)^2 < 2^24: every
    squared distance and every partial sum of one is then an integer below 2^24,
    exact in float32 in any summation order, so the GPU-assisted build writes the
    host builder's file byte for byte."""
    x = np.asarray(vectors)
    if x.ndim != 2 or x.size == 0:
        return False
    span = float(x.max()) - float(x.min())
    if x.shape[1] * span * span >= float(1 << 24):
        return False
    return all(np.array_equal(c, np.rint(c)) for c in np.array_split(x, max(1, x.shape[0] // 65536)))


def build_index(vectors: np.ndarray, attrs: np.ndarray, path: str, S: int, M: int, efc: int,
                seed: int = 0, threads: int = 0, device: int = 0) -> str:
    """Writes the HSIG of (vectors, attrs) to ``path``: GPU-assisted within the
    assist's limits (M <= 32, efc <= 256, d <= 1024, S <= 32), otherwise with the
    host builder. On data where assisted_build_is_exact holds the assisted file is the
    host builder's byte for byte; on other data the float32 distances of the two
    builders round differently, so a few neighbour choices can differ, and the graph
    is an equally valid HSIG (same levels, segments and attribute order)."""
    import hsig_build
    if M <= 32 and efc <= 256 and S <= 32 and np.asarray(vectors).shape[1] <= 1024:
        return build_index_gpu(vectors, attrs, path, S, M, efc, seed=seed, threads=threads, device=device)
    return hsig_build.build_index(vectors, attrs, path, S, M, efc, seed=seed, threads=threads)
