"""unify_search_noalloc: the search for callers that cannot allocate device memory
while searching (a fixed memory budget, or a latency-critical loop that cannot take
cudaMalloc's implicit synchronisation). It must return what unify_search returns,
call after call, from its fixed shared scratch array, and refuse sizes above its
limits. This file is named to be collected last."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

_P = ctypes.c_void_p


@pytest.fixture(scope="module")
def U():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2412_02448_gb300 as U
    assert torch.cuda.is_available()
    L = U.lib()
    L.unify_search_noalloc.argtypes = [_P, _P, _P, _P, ctypes.c_int64, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                       _P, _P, _P, _P, _P, _P]
    L.unify_search_noalloc.restype = ctypes.c_int
    return U


def _outputs(dev, nq, k):
    return dict(ids=torch.full((nq, k), -7, dtype=torch.int64, device=dev),
                dist=torch.full((nq, k), -7.0, dtype=torch.float32, device=dev),
                count=torch.full((nq,), -7, dtype=torch.int32, device=dev),
                status=torch.full((nq,), -7, dtype=torch.int32, device=dev))


def _noalloc(U, ix, q, lo, hi, k, ef, strategy, params, out=None):
    dev = ix.device
    q = torch.as_tensor(q, device=dev).contiguous()
    lo = torch.as_tensor(lo, device=dev).contiguous()
    hi = torch.as_tensor(hi, device=dev).contiguous()
    nq = q.shape[0]
    out = out if out is not None else _outputs(dev, nq, k)
    pp = lambda t: ctypes.c_void_p(t.data_ptr())
    rc = U.lib().unify_search_noalloc(ix._h, pp(q), pp(lo), pp(hi), nq, k, ef, U.STRATEGIES[strategy],
                                      ctypes.byref(params), pp(out["ids"]), pp(out["dist"]), pp(out["count"]),
                                      pp(out["status"]), ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream))
    torch.cuda.synchronize()
    return rc, {kk: v.cpu().numpy() for kk, v in out.items()}


def test_noalloc_matches_search_twice(U, c2_small_index):
    w, path = c2_small_index
    ix = U.Index(path)
    ta, tb = w.n // 100, w.n // 2
    params = U.Params.defaults(tau_a=ta, tau_b=tb)
    # two calls in a row per strategy, different batches (the second smaller), so
    # stale scratch contents from the first call would show
    batches = [(0, len(w.lo)), (7, 7 + 61)]
    for strategy in ("auto", "pre", "hybrid", "post"):
        for s, e in batches:
            Q, lo, hi = w.queries[s:e], w.lo[s:e], w.hi[s:e]
            rc, got = _noalloc(U, ix, Q, lo, hi, w.k, 64, strategy, params)
            assert rc == 0, U.lib().unify_last_error().decode()
            ref = ix.search(Q, lo, hi, w.k, ef=64, strategy=strategy, params=params)
            torch.cuda.synchronize()
            ref = {kk: v.cpu().numpy() for kk, v in ref.items()}
            # integer-valued vectors: float32 distances are exact, so equal bit for bit
            assert np.array_equal(got["ids"], ref["ids"]), strategy
            assert np.array_equal(got["count"], ref["count"]), strategy
            assert np.array_equal(got["dist"], ref["dist"]), strategy
            assert np.array_equal(got["status"], ref["status"]), strategy


def test_noalloc_rejects_sizes_above_its_limits(U, c2_small_index):
    w, path = c2_small_index
    ix = U.Index(path)
    params = U.Params.defaults()
    big = np.repeat(w.queries[:1], 1025, axis=0)
    rc, _ = _noalloc(U, ix, big, np.zeros(1025, np.int64), np.full(1025, 10**6, np.int64), 10, 64, "auto", params)
    assert rc == -6 and b"1024" in U.lib().unify_last_error()
    rc, _ = _noalloc(U, ix, w.queries[:4], w.lo[:4], w.hi[:4], 17, 64, "auto", params)
    assert rc == -6 and b"k must be" in U.lib().unify_last_error()


def test_noalloc_bf16_rerank_and_the_size_limits(U, c2_small_index):
    """At the limits (nq = 1024 queries, k = 16): BF16 storage with its FP32 re-rank of
    rerank_mult * k = 16 candidates, and pre-filter ranges split into the most scan
    items a query can have, equal unify_search (BF16 is exact on these integer
    coordinates, so bit for bit)."""
    w, path = c2_small_index
    ix = U.Index(path)
    ta, tb = w.n // 100, w.n // 2
    nq, k = 1024, 16
    sel = np.arange(nq) % len(w.lo)
    Q, lo, hi = w.queries[sel], w.lo[sel].copy(), w.hi[sel].copy()
    lo[::4], hi[::4] = -1, 10**7  # every object: the longest scans
    cases = [("auto", U.Params.defaults(dtype=U.BF16, rerank_mult=1, tau_a=ta, tau_b=tb)),
             ("pre", U.Params.defaults(scan_rows=96, tau_a=ta, tau_b=tb))]
    for strategy, params in cases:
        for _ in range(2):
            rc, got = _noalloc(U, ix, Q, lo, hi, k, 64, strategy, params)
            assert rc == 0, U.lib().unify_last_error().decode()
            ref = ix.search(Q, lo, hi, k, ef=64, strategy=strategy, params=params)
            torch.cuda.synchronize()
            ref = {kk: v.cpu().numpy() for kk, v in ref.items()}
            for key in ("ids", "dist", "count", "status"):
                assert np.array_equal(got[key], ref[key]), (strategy, key)
    rc, _ = _noalloc(U, ix, Q[:4], lo[:4], hi[:4], 16, 64, "auto", U.Params.defaults(dtype=U.BF16, rerank_mult=2))
    assert rc == -6 and b"rerank_mult * k" in U.lib().unify_last_error()


def test_noalloc_allocates_no_device_memory(U, c2_small_index):
    """On a freshly loaded index, whose own scratch has never been grown, a call leaves
    the device's free memory unchanged."""
    w, path = c2_small_index
    ix0 = U.Index(path)
    rc, _ = _noalloc(U, ix0, w.queries[:8], w.lo[:8], w.hi[:8], w.k, 64, "auto", U.Params.defaults())
    assert rc == 0
    ix = U.Index(path)
    Q, lo, hi = (torch.as_tensor(a, device=ix.device).contiguous() for a in (w.queries, w.lo, w.hi))
    out = _outputs(ix.device, len(w.lo), w.k)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info(ix.device)[0]
    rc, got = _noalloc(U, ix, Q, lo, hi, w.k, 64, "auto", U.Params.defaults(tau_a=w.n // 100, tau_b=w.n // 2),
                       out=out)
    free1 = torch.cuda.mem_get_info(ix.device)[0]
    assert rc == 0 and free1 == free0
    assert np.all(got["count"] >= 0)
