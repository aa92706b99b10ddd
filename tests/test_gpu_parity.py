"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Integer-valued vectors (the c2 shape: coordinates in [0, 255], d = 128) make
every float32 squared distance an exact integer below 2**24, so the GPU's
float32 arithmetic equals the oracle's FP64 exactly and the approximate
strategies must follow the very same traversal: ids and expansion counts are
compared bit for bit. On real-valued data (c1) the pre-filter ids may only
differ by swaps of items whose FP64 distances lie within 2e-5 relative, and
distances must be within 1e-5 relative of FP64.
"""
import json
import os

import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
EXACT_BITS = 3  # UNIFY_Q_LIMIT | UNIFY_Q_TRUNCATED
CAND = 4096     # candidate-buffer entries used by the exactness checks (the maximum)


def _exact_rows(r, o, cap=CAND, floor=0.98, what=""):
    """Rows to compare bit for bit, after checking that every flag is legitimate.

    The candidate buffer holds visited objects only, so a row can overflow it
    (UNIFY_Q_TRUNCATED) only when its exact traversal visits more objects than the
    buffer holds: the oracle's distance count, summed over all layers, is an upper
    bound. The expansion bound (100,000 per layer, UNIFY_Q_LIMIT) is out of reach at
    these sizes. Flagged rows are reported with their recall against the oracle's
    traversal; at least ``floor`` of the rows must be unflagged."""
    st = r["status"]
    assert not np.any(st & 1), what  # UNIFY_Q_LIMIT
    trunc = (st & 2) != 0
    assert np.all(o["n_dist"][trunc] > cap), (what, np.flatnonzero(trunc & (o["n_dist"] <= cap)))
    ok = ~trunc
    if trunc.any():
        k = r["ids"].shape[1]
        rec = oracle.recall(r["ids"][trunc], o["ids"][trunc], o["count"][trunc], k)
        print(f"{what}: {trunc.mean():.3f} of rows truncated; their recall against the oracle's rows "
              f"{rec.mean():.3f} (min {rec.min():.3f})")
    assert ok.mean() >= floor, (what, ok.mean())
    return ok


def _valid(w, r, lo, hi):
    """Invariants of any result row: ids in range, no duplicates, sorted, padded."""
    for i in range(len(lo)):
        c = int(r["count"][i])
        ids = r["ids"][i, :c]
        assert np.all((w.attrs[ids] >= lo[i]) & (w.attrs[ids] <= hi[i]))
        assert len(set(ids.tolist())) == c and np.all(r["ids"][i, c:] == -1)
        keys = list(zip(r["dist"][i, :c].tolist(), ids.tolist()))
        assert keys == sorted(keys)


@pytest.fixture(scope="module")
def U():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2412_02448_gb300 as U
    assert torch.cuda.is_available()
    return U


def _np(r):
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in r.items()}


def _edge_ranges(w):
    lo = np.array([-5, 10**9, 7, 500, 0, -(2**62), 123456], np.int64)
    hi = np.array([-1, 10**9 + 5, 6, 500, 10**7, 2**62, 123456 + 1000], np.int64)
    q = w.queries[: len(lo)]
    return q, lo, hi


def test_route_parity(U, c2_small_index, c1_index):
    for w, path in (c2_small_index, c1_index):
        ix = U.Index(path)
        oi = oracle.OracleIndex(path)
        q, elo, ehi = _edge_ranges(w)
        lo = np.concatenate([w.lo, elo])
        hi = np.concatenate([w.hi, ehi])
        ta, tb = w.n // 100, w.n // 2
        g = _np(ix.route(lo, hi, ta, tb))
        o = oi.route(lo, hi, ta, tb)
        assert np.array_equal(g["pa"], o["pa"]) and np.array_equal(g["pb"], o["pb"])
        assert np.array_equal(g["mask"].astype(np.uint32), o["mask"])
        assert np.array_equal(g["strategy"], o["strategy"])


def test_prefilter_exact_integer_data(U, c2_small_index):
    w, path = c2_small_index
    ix = U.Index(path)
    q, elo, ehi = _edge_ranges(w)
    Q = np.concatenate([w.queries, q])
    lo = np.concatenate([w.lo, elo])
    hi = np.concatenate([w.hi, ehi])
    ex_ids, ex_d, ex_c = oracle.exact_knn(w.vectors, w.attrs, Q, lo, hi, w.k)
    for scan_rows in (8192, 96):  # one work item, and a ragged split merged by the second kernel
        r = _np(ix.search(Q, lo, hi, w.k, strategy="pre", params=U.Params.defaults(scan_rows=scan_rows),
                          counters=True))
        assert np.array_equal(r["count"], ex_c)
        assert np.array_equal(r["ids"], ex_ids)
        fin = np.isfinite(ex_d)
        assert np.array_equal(r["dist"][fin].astype(np.float64), ex_d[fin])
        assert np.all(np.isinf(r["dist"][~fin]))


def test_prefilter_tie_band_real_data(U, c1_index):
    w, path = c1_index
    ix = U.Index(path)
    for k in (1, 10, 100):
        ex_ids, ex_d, ex_c = oracle.exact_knn(w.vectors, w.attrs, w.queries, w.lo, w.hi, k)
        r = _np(ix.search(w.queries, w.lo, w.hi, k, strategy="pre"))
        assert np.array_equal(r["count"], ex_c)
        for i in range(len(w.lo)):
            c = ex_c[i]
            g, e = r["ids"][i, :c], ex_ids[i, :c]
            gd = r["dist"][i, :c].astype(np.float64)
            assert np.all(np.abs(gd - ex_d[i, :c]) <= 1e-5 * np.maximum(ex_d[i, :c], 1e-30))
            if not np.array_equal(g, e):
                # only swaps inside the FP64 tie band, including at the k-th boundary
                X = w.vectors.astype(np.float64)
                dg = ((X[g] - w.queries[i].astype(np.float64)) ** 2).sum(1)
                kth = ex_d[i, c - 1]
                assert np.all(dg <= kth * (1 + 2e-5))
                diff = set(g.tolist()) ^ set(e.tolist())
                X_d = {j: ((X[j] - w.queries[i].astype(np.float64)) ** 2).sum() for j in diff}
                assert all(abs(X_d[j] - kth) <= 2e-5 * kth for j in diff)


@pytest.mark.parametrize("strategy", ["hybrid", "post"])
@pytest.mark.parametrize("ef", [10, 64, 200])
def test_graph_strategies_match_oracle(U, c2_small_index, strategy, ef):
    """Same traversal as the oracle's literal Algorithms 1/2/7: ids and expansion
    counts identical wherever the GPU reports no truncation or expansion limit."""
    w, path = c2_small_index
    ix = U.Index(path)
    oi = oracle.OracleIndex(path)
    r = _np(ix.search(w.queries, w.lo, w.hi, w.k, ef=ef, strategy=strategy, counters=True,
                      params=U.Params.defaults(cand_cap=CAND)))
    o = oi.search(w.queries, w.lo, w.hi, w.k, ef=ef, m=16, strategy=strategy)
    _valid(w, r, w.lo, w.hi)
    ok = _exact_rows(r, o, what=f"{strategy} ef={ef}")
    # every row's exact traversal fits the buffer here, so every row is compared
    assert np.all(o["n_dist"] <= CAND) and ok.all()
    assert np.array_equal(r["ids"][ok], o["ids"][ok])
    assert np.array_equal(r["count"][ok], o["count"][ok])
    assert np.array_equal(r["counters"][ok, 1], o["n_exp"][ok])
    fin = np.isfinite(o["dist"][ok])
    assert np.array_equal(r["dist"][ok][fin].astype(np.float64), o["dist"][ok][fin])


@pytest.mark.parametrize("m", [4, 16, 40])
def test_hybrid_selection_width(U, c2_small_index, m):
    w, path = c2_small_index
    ix = U.Index(path)
    oi = oracle.OracleIndex(path)
    r = _np(ix.search(w.queries, w.lo, w.hi, w.k, ef=50, strategy="hybrid",
                      params=U.Params.defaults(m=m, cand_cap=CAND), counters=True))
    o = oi.search(w.queries, w.lo, w.hi, w.k, ef=50, m=m, strategy="hybrid")
    _valid(w, r, w.lo, w.hi)
    ok = _exact_rows(r, o, what=f"hybrid m={m}")
    assert np.all(o["n_dist"] <= CAND) and ok.all()
    assert np.array_equal(r["ids"][ok], o["ids"][ok])
    assert np.array_equal(r["counters"][ok, 1], o["n_exp"][ok])


def test_auto_routing_matches_oracle(U, c2_small_index):
    w, path = c2_small_index
    ix = U.Index(path)
    oi = oracle.OracleIndex(path)
    ta, tb = w.n // 100, w.n // 2
    p = U.Params.defaults(tau_a=ta, tau_b=tb, cand_cap=CAND)
    r = _np(ix.search(w.queries, w.lo, w.hi, w.k, ef=80, strategy="auto", params=p))
    _valid(w, r, w.lo, w.hi)
    o = oi.search(w.queries, w.lo, w.hi, w.k, ef=80, m=16, strategy="auto", tau_a=ta, tau_b=tb)
    assert set(np.unique(o["strategy"]).tolist()) == {0, 1, 2}
    ok = _exact_rows(r, o, what="auto")
    assert ok.all()
    assert np.array_equal(r["ids"][ok], o["ids"][ok])
    assert np.array_equal(r["count"], o["count"])
    ex = oracle.exact_knn(w.vectors, w.attrs, w.queries, w.lo, w.hi, w.k)
    rec = oracle.recall(r["ids"], ex[0], ex[2], w.k)
    assert rec.mean() > 0.9


@pytest.mark.parametrize("name", ["tiny_line_graph", "layered_line_graph"])
def test_golden_graphs_gpu(U, tmp_path, name):
    """The hand-traced cases of the one-layer and the three-layer golden indexes
    through the C ABI: ids, distances and expansion counts as traced (the upper
    layers' entry points show in the expansion counts); the GPU counts at least the
    traced distance evaluations (a forgotten visited id is evaluated again). Range
    bounds and masks of the layered index's route cases as traced."""
    from index_writer import layered_index_sections, tiny_index_sections, write_index
    with open(os.path.join(GOLDEN, name + ".json")) as f:
        g = json.load(f)
    path = str(tmp_path / (name + ".idx"))
    write_index(path, (layered_index_sections if "upper" in g else tiny_index_sections)(g))
    ix = U.Index(path)
    if "route_cases" in g:
        rc = g["route_cases"]
        rt = _np(ix.route(np.array([c["lo"] for c in rc]), np.array([c["hi"] for c in rc])))
        for i, c in enumerate(rc):
            assert (int(rt["pa"][i]), int(rt["pb"][i]), int(rt["mask"][i])) == (c["pa"], c["pb"], c["mask"]), c
    for case in g["cases"]:
        p = U.Params.defaults(m=case["m"], ef_post=case["ef"])
        r = _np(ix.search(np.array([case["q"]], np.float32), [case["lo"]], [case["hi"]], case["k"],
                          ef=case["ef"], strategy=case["strategy"], params=p, counters=True))
        assert list(r["ids"][0]) == case["expect_ids"], case["name"]
        for got, exp in zip(r["dist"][0], case["expect_dist"]):
            if exp is None:
                assert np.isinf(got)
            else:
                assert got == pytest.approx(exp, rel=1e-5, abs=1e-6)
        if case["strategy"] != "pre":
            assert r["counters"][0, 1] == case["expect_n_exp"], case["name"]
            # the oracle evaluates each layer's entry point again; the GPU carries its
            # key down from the layer above (one evaluation fewer per layer below the top)
            reused = max(g.get("level", [0]))
            assert r["counters"][0, 0] >= case["expect_n_dist"] - reused, case["name"]


def test_edge_cases(U, c2_small_index):
    w, path = c2_small_index
    ix = U.Index(path)
    # empty batch
    r = ix.search(np.zeros((0, w.d), np.float32), np.zeros(0, np.int64), np.zeros(0, np.int64), 5)
    assert r["ids"].shape == (0, 5)
    # k = 1 and k = 256 (the maximum), k above |R|
    lo = np.array([w.lo[0], 5, 100], np.int64)
    hi = np.array([w.hi[0], 4, 160], np.int64)  # second is lo > hi
    for k in (1, 256):
        for st in ("pre", "hybrid", "post"):
            r = _np(ix.search(w.queries[:3], lo, hi, k, ef=300, strategy=st))
            assert r["count"][1] == 0 and np.all(r["ids"][1] == -1)
            for i in (0, 2):
                c = r["count"][i]
                ids = r["ids"][i, :c]
                assert np.all((w.attrs[ids] >= lo[i]) & (w.attrs[ids] <= hi[i]))
                assert len(set(ids.tolist())) == c and np.all(r["ids"][i, c:] == -1)
    # invalid arguments are reported, not run
    with pytest.raises(U.UnifyError):
        ix.search(w.queries[:2], w.lo[:2], w.hi[:2], 0)
    with pytest.raises(U.UnifyError):
        ix.search(w.queries[:2], w.lo[:2], w.hi[:2], 257)
    with pytest.raises(U.UnifyError):
        ix.search(w.queries[:2], w.lo[:2], w.hi[:2], 10, params=U.Params.defaults(visited_cap=1000))


def test_host_buffers_equal_device(U, c2_small_index):
    w, path = c2_small_index
    ix = U.Index(path)
    ta, tb = w.n // 100, w.n // 2
    p = U.Params.defaults(tau_a=ta, tau_b=tb)
    d = _np(ix.search(w.queries, w.lo, w.hi, w.k, ef=64, strategy="auto", params=p))
    h = ix.search_auto_host(w.queries, w.lo, w.hi, w.k, ef=64, params=p)
    assert np.array_equal(d["ids"], h["ids"]) and np.array_equal(d["count"], h["count"])


def test_bad_index_files_rejected(U, tmp_path):
    from index_writer import tiny_index_sections, write_index
    with open(os.path.join(GOLDEN, "tiny_line_graph.json")) as f:
        g = json.load(f)
    sec = tiny_index_sections(g)
    bad = str(tmp_path / "bad.idx")
    write_index(bad, sec, corrupt_section="vectors")
    with pytest.raises(U.UnifyError, match="checksum"):
        U.Index(bad)
    sec2 = dict(sec)
    adj = sec["adj0"].copy()
    adj[0, 0, 0] = 10**6  # neighbour id out of range
    sec2["adj0"] = adj
    write_index(bad, sec2)
    with pytest.raises(U.UnifyError, match="out of range"):
        U.Index(bad)
    with pytest.raises(U.UnifyError):
        U.Index(str(tmp_path / "missing.idx"))
    # wrong magic, unsupported version, truncated file
    write_index(bad, sec)
    raw = bytearray(open(bad, "rb").read())
    for name, data in (("magic", bytes([raw[0] ^ 0xFF]) + bytes(raw[1:])),
                       ("version", bytes(raw[:8]) + (2).to_bytes(4, "little") + bytes(raw[12:])),
                       ("truncated", bytes(raw[: len(raw) // 2]))):
        path = str(tmp_path / f"{name}.idx")
        with open(path, "wb") as f:
            f.write(data)
        with pytest.raises(U.UnifyError):
            U.Index(path)


def test_cuda_graph_plan_replays_search(U, c2_small_index):
    w, path = c2_small_index
    ix = U.Index(path)
    ta, tb = w.n // 100, w.n // 2
    p = U.Params.defaults(tau_a=ta, tau_b=tb)
    nq = 200
    plan = ix.plan(w.queries[:nq], w.lo[:nq], w.hi[:nq], w.k, ef=64, params=p)
    for shift in (0, 100):
        # update the captured input buffers in place, then replay
        plan.q.copy_(torch.from_numpy(w.queries[shift:shift + nq]))
        plan.lo.copy_(torch.from_numpy(w.lo[shift:shift + nq]))
        plan.hi.copy_(torch.from_numpy(w.hi[shift:shift + nq]))
        got = _np(plan.launch())
        ref = _np(ix.search(w.queries[shift:shift + nq], w.lo[shift:shift + nq], w.hi[shift:shift + nq], w.k,
                            ef=64, params=p))
        assert np.array_equal(got["ids"], ref["ids"]) and np.array_equal(got["count"], ref["count"])
        assert np.array_equal(got["dist"], ref["dist"])
    # a search needing more scratch than the plan holds is refused while the plan lives
    big = np.repeat(w.queries[:1], 300_000, axis=0)
    with pytest.raises(U.UnifyError, match="plan"):
        ix.search(big, np.zeros(len(big), np.int64), np.zeros(len(big), np.int64), w.k)
    plan.close()
    r = ix.search(big[:5000], np.zeros(5000, np.int64), np.zeros(5000, np.int64), w.k)
    torch.cuda.synchronize()


@pytest.mark.parametrize("strategy", ["pre", "hybrid", "post", "auto"])
def test_bf16_storage_lossless_on_integer_data(U, c2_small_index, strategy):
    """Coordinates 0..255 are exact in bfloat16, so the BF16 traversal and scan see
    the FP32 distances and the FP32 re-rank returns the FP32 path's rows exactly."""
    w, path = c2_small_index
    ix = U.Index(path)
    ta, tb = w.n // 100, w.n // 2
    base = dict(tau_a=ta, tau_b=tb, cand_cap=CAND)
    for scan_rows in (8192, 96):
        f32 = _np(ix.search(w.queries, w.lo, w.hi, w.k, ef=48, strategy=strategy,
                            params=U.Params.defaults(scan_rows=scan_rows, **base)))
        b16 = _np(ix.search(w.queries, w.lo, w.hi, w.k, ef=48, strategy=strategy,
                            params=U.Params.defaults(dtype=U.BF16, rerank_mult=4, scan_rows=scan_rows, **base)))
        for key in ("ids", "dist", "count", "status"):
            assert np.array_equal(f32[key], b16[key]), (strategy, key)


@pytest.mark.parametrize("dataset", ["c2_small_index", "c1_index"])
def test_fp8_storage_rerank(U, dataset, request):
    """FP8 E4M3 with a per-vector scale is lossy; after the FP32 re-rank every
    returned distance is the float32 direct distance of that id (within 1e-5 of
    FP64) and recall stays high."""
    w, path = request.getfixturevalue(dataset)
    ix = U.Index(path)
    ta, tb = w.n // 100, w.n // 2
    X = w.vectors.astype(np.float64)
    ex = oracle.exact_knn(w.vectors, w.attrs, w.queries, w.lo, w.hi, w.k)
    for dtype in (U.FP8E4M3, U.BF16):
        for strategy in ("pre", "auto"):
            p = U.Params.defaults(dtype=dtype, rerank_mult=4, tau_a=ta, tau_b=tb, m=32, cand_cap=CAND)
            r = _np(ix.search(w.queries, w.lo, w.hi, w.k, ef=96, strategy=strategy, params=p))
            _valid(w, r, w.lo, w.hi)
            for i in range(len(w.lo)):
                c = r["count"][i]
                ids = r["ids"][i, :c]
                d64 = ((X[ids] - w.queries[i].astype(np.float64)) ** 2).sum(1)
                assert np.all(np.abs(r["dist"][i, :c] - d64) <= 1e-5 * np.maximum(d64, 1e-30))
            rec = oracle.recall(r["ids"], ex[0], ex[2], w.k)
            floor = 0.97 if strategy == "pre" else 0.85
            assert rec.mean() >= floor, (dataset, dtype, strategy, rec.mean())


def test_register_budgets_give_identical_results(U, c1_index):
    """The 128/80/64-register variants differ in distance-group size only; every
    vector's distance uses the same lane order and reduction tree, so with the same
    buffer sizes every row (flagged ones included) is bit-identical on real data."""
    w, path = c1_index
    ix = U.Index(path)
    ta, tb = w.n // 100, w.n // 2
    for strategy in ("auto", "hybrid", "post"):
        ref = None
        for regs in (128, 80, 64):
            p = U.Params.defaults(tau_a=ta, tau_b=tb, reg_budget=regs, visited_cap=1024, cand_cap=512)
            r = _np(ix.search(w.queries, w.lo, w.hi, w.k, ef=64, strategy=strategy, params=p, counters=True))
            if ref is None:
                ref = r
                continue
            for key in ("ids", "dist", "count", "status"):
                assert np.array_equal(r[key], ref[key]), (regs, strategy, key)
            assert np.array_equal(r["counters"][:, :2], ref["counters"][:, :2]), (regs, strategy)


@pytest.mark.parametrize("dataset", ["c3_small_index", "c5_small_index"])
def test_other_widths_real_data(U, dataset, request):
    """d = 96 (one partial chunk per lane) and d = 960 (eight chunks per lane, the
    widest kernel variant) on real-valued data: the exact pre-filter within the FP64
    tie band, distances within 1e-5 of FP64, graph strategies valid with high recall,
    and every storage format."""
    w, path = request.getfixturevalue(dataset)
    ix = U.Index(path)
    X = w.vectors.astype(np.float64)
    ex_ids, ex_d, ex_c = oracle.exact_knn(w.vectors, w.attrs, w.queries, w.lo, w.hi, w.k)
    ta, tb = w.n // 100, w.n // 2
    for dtype in (U.FP32, U.BF16, U.FP8E4M3):
        for strategy in ("pre", "auto", "hybrid", "post"):
            for regs in (128, 64):
                p = U.Params.defaults(dtype=dtype, tau_a=ta, tau_b=tb, m=32, cand_cap=CAND, reg_budget=regs,
                                      visited_cap=1024, scan_rows=512)
                r = _np(ix.search(w.queries, w.lo, w.hi, w.k, ef=128, strategy=strategy, params=p))
                _valid(w, r, w.lo, w.hi)
                for i in range(len(w.lo)):
                    c = r["count"][i]
                    ids = r["ids"][i, :c]
                    d64 = ((X[ids] - w.queries[i].astype(np.float64)) ** 2).sum(1)
                    assert np.all(np.abs(r["dist"][i, :c] - d64) <= 1e-5 * np.maximum(d64, 1e-30)), (dtype, strategy)
                rec = oracle.recall(r["ids"], ex_ids, ex_c, w.k)
                if strategy == "pre":
                    assert np.array_equal(r["count"], ex_c)
                    assert rec.mean() >= (0.999 if dtype == U.FP32 else 0.98), (dataset, dtype, regs, rec.mean())
                elif strategy == "auto":
                    # forced post-filtering on narrow ranges is poor by design (the
                    # paper's motivation for routing); the routed batch must be good
                    assert rec.mean() >= 0.85, (dataset, dtype, regs, rec.mean())


@pytest.mark.parametrize("dtype", ["BF16", "FP32"])
def test_tensor_core_scan_equals_exact_answer(U, c2_small_index, dtype):
    """The tcgen05 pre-filter scan (MMA over row tiles shared by 128 queries, bfloat16
    operands for BF16 storage, tf32 for FP32 storage, then the FP32 re-rank) returns the
    oracle's exact answer (Definition 1, FP64) id for id and distance for distance on
    integer data, whose values are exact in both operand formats: ragged tiles (300,
    129, 65 and 1 queries), several work units per tile, and re-rank widths R = k, 4k,
    6k, and the widest sets (R = 64 at k = 32 and 64, R = k = 100 and 128). In a routed batch the tensor-core phase takes the pre-filter queries and the
    search kernel the others, and every row equals the oracle's HSIG search."""
    w, path = c2_small_index
    ix = U.Index(path)
    dt = getattr(U, dtype)
    for nq in (len(w.lo), 129, 65, 1):
        Q, lo, hi = w.queries[:nq], w.lo[:nq], w.hi[:nq]
        ex_ids, ex_d, ex_c = oracle.exact_knn(w.vectors, w.attrs, Q, lo, hi, w.k)
        fin = np.isfinite(ex_d)
        for rm in (1, 4, 6):
            tc = _np(ix.search(Q, lo, hi, w.k, strategy="pre",
                               params=U.Params.defaults(dtype=dt, rerank_mult=rm, tc_scan=1)))
            assert np.array_equal(tc["ids"], ex_ids), (dtype, nq, rm)
            assert np.array_equal(tc["count"], ex_c), (dtype, nq, rm)
            assert np.array_equal(tc["dist"][fin].astype(np.float64), ex_d[fin]), (dtype, nq, rm)
            assert np.all(np.isinf(tc["dist"][~fin])) and np.all(tc["status"] == 0)
    # the widest candidate sets the scan keeps (R = rerank_mult * k up to 64, else k,
    # up to 128: there the bound is the largest group minimum, and lists overflow into
    # the exact warp scan of the query's range)
    for k, rm in ((100, 1), (100, 4), (64, 2), (32, 4), (128, 1)):
        Q, lo, hi = w.queries[:129], w.lo[:129], w.hi[:129]
        ex_ids, ex_d, ex_c = oracle.exact_knn(w.vectors, w.attrs, Q, lo, hi, k)
        fin = np.isfinite(ex_d)
        tc = _np(ix.search(Q, lo, hi, k, strategy="pre", params=U.Params.defaults(dtype=dt, rerank_mult=rm, tc_scan=1)))
        assert np.array_equal(tc["ids"], ex_ids), (dtype, k, rm)
        assert np.array_equal(tc["count"], ex_c), (dtype, k, rm)
        assert np.array_equal(tc["dist"][fin].astype(np.float64), ex_d[fin]), (dtype, k, rm)
    ta, tb = w.n // 20, w.n // 2
    p1 = U.Params.defaults(dtype=dt, rerank_mult=4, tau_a=ta, tau_b=tb, cand_cap=CAND, tc_scan=1)
    r1 = _np(ix.search(w.queries, w.lo, w.hi, w.k, ef=64, strategy="auto", params=p1))
    o = oracle.OracleIndex(path).search(w.queries, w.lo, w.hi, w.k, ef=64, m=16, strategy="auto", tau_a=ta,
                                        tau_b=tb)
    assert set(np.unique(o["strategy"]).tolist()) == {0, 1, 2}
    assert np.array_equal(r1["ids"], o["ids"]) and np.array_equal(r1["count"], o["count"])
    fin = np.isfinite(o["dist"])
    assert np.array_equal(r1["dist"][fin].astype(np.float64), o["dist"][fin])


def test_tensor_core_scan_wait_timeout_recovers(U, c2_small_index):
    """The tensor-core scan's failure path, without a GPU fault: with tc_scan = 2 the
    collecting pass waits on a barrier that nothing arrives at, under a 50 ms limit.
    The wait runs out, the other roles' waits run out in turn and drain, and the call
    returns normally with every pre-filter row empty and flagged UNIFY_Q_LIMIT, while
    the graph-routed rows of the same batch are searched as usual. The next search on
    the same index returns the warp scan's rows again."""
    w, path = c2_small_index
    ix = U.Index(path)
    ta, tb = w.n // 100, w.n // 2
    ref = _np(ix.search(w.queries, w.lo, w.hi, w.k, ef=64, strategy="auto",
                        params=U.Params.defaults(dtype=U.BF16, rerank_mult=4, tau_a=ta, tau_b=tb, cand_cap=CAND)))
    pre = oracle.OracleIndex(path).route(w.lo, w.hi, ta, tb)["strategy"] == 0
    assert 0 < pre.sum() < len(pre)
    bad = _np(ix.search(w.queries, w.lo, w.hi, w.k, ef=64, strategy="auto",
                        params=U.Params.defaults(dtype=U.BF16, rerank_mult=4, tau_a=ta, tau_b=tb, cand_cap=CAND,
                                                 tc_scan=2)))
    assert np.all((bad["status"][pre] & U.Q_LIMIT) != 0)
    assert np.all(bad["count"][pre] == 0) and np.all(bad["ids"][pre] == -1)
    for key in ("ids", "dist", "count", "status"):
        assert np.array_equal(bad[key][~pre], ref[key][~pre]), key
    again = _np(ix.search(w.queries, w.lo, w.hi, w.k, ef=64, strategy="auto",
                          params=U.Params.defaults(dtype=U.BF16, rerank_mult=4, tau_a=ta, tau_b=tb, cand_cap=CAND,
                                                   tc_scan=1)))
    for key in ("ids", "dist", "count", "status"):
        assert np.array_equal(again[key], ref[key]), key
    with pytest.raises(U.UnifyError):
        ix.search(w.queries[:4], w.lo[:4], w.hi[:4], w.k, params=U.Params.defaults(tc_scan=3))


@pytest.mark.parametrize("dtype", ["BF16", "FP32", "FP8E4M3"])
def test_tensor_core_scan_wide_rows(U, c5_small_index, dtype):
    """d = 960 (K-slices of 64, 32 or 128 elements per stage) on real data: the
    candidates are chosen by the expanded distance form over the operand format, so
    rows may differ from the exact scan only by near-ties; every returned distance is
    the float32 distance of its id (within 1e-4 relative of FP64, d = 960 terms), and
    recall against the exact answer is near 1 (0.97 for E4M3, whose 3-bit mantissa
    blurs the candidates' order more)."""
    w, path = c5_small_index
    ix = U.Index(path)
    X = w.vectors.astype(np.float64)
    ex = oracle.exact_knn(w.vectors, w.attrs, w.queries, w.lo, w.hi, w.k)
    r = _np(ix.search(w.queries, w.lo, w.hi, w.k, strategy="pre",
                      params=U.Params.defaults(dtype=getattr(U, dtype), rerank_mult=4, tc_scan=1)))
    _valid(w, r, w.lo, w.hi)
    assert np.array_equal(r["count"], np.minimum(ex[2], w.k))
    assert np.all(r["status"] == 0)
    for i in range(len(w.lo)):
        c = r["count"][i]
        ids = r["ids"][i, :c]
        d64 = ((X[ids] - w.queries[i].astype(np.float64)) ** 2).sum(1)
        assert np.all(np.abs(r["dist"][i, :c] - d64) <= 1e-4 * np.maximum(d64, 1e-30))
    rec = oracle.recall(r["ids"], ex[0], ex[2], w.k)
    assert rec.mean() >= (0.97 if dtype == "FP8E4M3" else 0.99), (dtype, rec.mean())


@pytest.mark.parametrize("m", [4, 12, 40])
def test_hybrid_s1_matches_oracle(U, c2_small_index, m):
    """Selection S1 (the m neighbours nearest to the expanded object over all
    intersected chunks). On integer data every owner distance is an exact integer in
    float32, so the GPU selects the oracle's neighbours and follows its traversal:
    ids, distances, counts and expansion counts identical on unflagged rows; BF16
    storage (exact on this data) gives the same rows; m above 64 is refused."""
    w, path = c2_small_index
    ix = U.Index(path)
    oi = oracle.OracleIndex(path)
    p = U.Params.defaults(m=m, cand_cap=CAND, selection=1)
    r = _np(ix.search(w.queries, w.lo, w.hi, w.k, ef=50, strategy="hybrid", params=p, counters=True))
    o = oi.search(w.queries, w.lo, w.hi, w.k, ef=50, m=m, strategy="hybrid", selection=1)
    _valid(w, r, w.lo, w.hi)
    ok = _exact_rows(r, o, what=f"S1 m={m}")
    assert np.all(o["n_dist"] <= CAND) and ok.all()
    assert np.array_equal(r["ids"][ok], o["ids"][ok])
    assert np.array_equal(r["count"][ok], o["count"][ok])
    assert np.array_equal(r["counters"][ok, 1], o["n_exp"][ok])
    fin = np.isfinite(o["dist"][ok])
    assert np.array_equal(r["dist"][ok][fin].astype(np.float64), o["dist"][ok][fin])
    # S1 differs from S2 on this data (the variant is really taken)
    s2 = oi.search(w.queries, w.lo, w.hi, w.k, ef=50, m=m, strategy="hybrid", selection=2)
    assert not np.array_equal(o["n_exp"], s2["n_exp"])
    b = _np(ix.search(w.queries, w.lo, w.hi, w.k, ef=50, strategy="hybrid", counters=True,
                      params=U.Params.defaults(m=m, cand_cap=CAND, selection=1, dtype=U.BF16, rerank_mult=4)))
    for key in ("ids", "dist", "count", "status"):
        assert np.array_equal(b[key], r[key]), key
    with pytest.raises(U.UnifyError):
        ix.search(w.queries, w.lo, w.hi, w.k, ef=50, strategy="hybrid",
                  params=U.Params.defaults(m=65, selection=1))


def test_conjunctive_second_attribute_matches_oracle(U, c2_small_index):
    """Conjunctive queries (a second attribute, Section 5.9): the pre-filter equals the
    exact conjunctive answer; hybrid and post-filter follow the oracle's traversal
    (ids, distances, counts and expansion counts on unflagged rows); auto routing
    agrees; a second range that holds every object gives the plain search's rows."""
    from workloads import second_attribute
    w, path = c2_small_index
    ix = U.Index(path)
    oi = oracle.OracleIndex(path)
    fr = np.array([0.2, 0.5, 1.0])[np.arange(len(w.lo)) % 3]
    a2, lo2, hi2 = second_attribute(w.n, fr, 11)
    ex = oracle.exact_knn(w.vectors, w.attrs, w.queries, w.lo, w.hi, w.k, attr2=a2, lo2=lo2, hi2=hi2)
    r = _np(ix.search(w.queries, w.lo, w.hi, w.k, strategy="pre", attr2=a2, lo2=lo2, hi2=hi2))
    assert np.array_equal(r["ids"], ex[0]) and np.array_equal(r["count"], ex[2])
    assert np.array_equal(r["dist"].astype(np.float64)[np.isfinite(ex[1])], ex[1][np.isfinite(ex[1])])
    ta, tb = w.n // 100, w.n // 2
    for strategy in ("hybrid", "post", "auto"):
        p = U.Params.defaults(cand_cap=CAND, tau_a=ta, tau_b=tb)
        r = _np(ix.search(w.queries, w.lo, w.hi, w.k, ef=64, strategy=strategy, params=p, counters=True,
                          attr2=a2, lo2=lo2, hi2=hi2))
        o = oi.search(w.queries, w.lo, w.hi, w.k, ef=64, m=16, strategy=strategy, tau_a=ta, tau_b=tb,
                      attr2=a2, lo2=lo2, hi2=hi2)
        ok = _exact_rows(r, o, what=f"conjunctive {strategy}")
        assert np.all(o["n_dist"] <= CAND) and ok.all(), strategy
        for i in np.flatnonzero(ok)[:50]:
            c = int(r["count"][i])
            ids = r["ids"][i, :c]
            assert np.all((w.attrs[ids] >= w.lo[i]) & (w.attrs[ids] <= w.hi[i]))
            assert np.all((a2[ids] >= lo2[i]) & (a2[ids] <= hi2[i]))
        assert np.array_equal(r["ids"][ok], o["ids"][ok]), strategy
        assert np.array_equal(r["count"][ok], o["count"][ok]), strategy
        graph = ok & (o["strategy"] != 0)
        assert np.array_equal(r["counters"][graph, 1], o["n_exp"][graph]), strategy
        fin = np.isfinite(o["dist"][ok])
        assert np.array_equal(r["dist"][ok][fin].astype(np.float64), o["dist"][ok][fin]), strategy
    full_lo = np.full(len(w.lo), -1, np.int64)
    full_hi = np.full(len(w.lo), 10**6, np.int64)
    p = U.Params.defaults(cand_cap=CAND, tau_a=ta, tau_b=tb)
    plain = _np(ix.search(w.queries, w.lo, w.hi, w.k, ef=64, strategy="auto", params=p))
    conj = _np(ix.search(w.queries, w.lo, w.hi, w.k, ef=64, strategy="auto", params=p, attr2=a2, lo2=full_lo,
                         hi2=full_hi))
    for key in ("ids", "dist", "count", "status"):
        assert np.array_equal(plain[key], conj[key]), key


@pytest.mark.parametrize("dtype", ["BF16", "FP32", "FP8E4M3"])
def test_tensor_core_scan_partial_slices_and_empty_ranges(U, c3_small_index, c2_small_index, dtype):
    """d = 96 (the last K-slice is partly outside the rows for bfloat16 and E4M3; TMA
    fills it with zeros): every returned distance is the float32 distance of its id,
    counts are exact and recall is near 1. Tiles that mix empty, reversed and one-row
    ranges with ordinary ones give the warp scan's rows on integer data (bfloat16 and
    tf32 operands; E4M3 codes are not exact there, so its rows are checked for valid
    distances and counts)."""
    w, path = c3_small_index
    ix = U.Index(path)
    dt = getattr(U, dtype)
    X = w.vectors.astype(np.float64)
    ex = oracle.exact_knn(w.vectors, w.attrs, w.queries, w.lo, w.hi, w.k)
    r = _np(ix.search(w.queries, w.lo, w.hi, w.k, strategy="pre",
                      params=U.Params.defaults(dtype=dt, rerank_mult=4, tc_scan=1)))
    _valid(w, r, w.lo, w.hi)
    assert np.array_equal(r["count"], np.minimum(ex[2], w.k)) and np.all(r["status"] == 0)
    for i in range(len(w.lo)):
        c = r["count"][i]
        ids = r["ids"][i, :c]
        d64 = ((X[ids] - w.queries[i].astype(np.float64)) ** 2).sum(1)
        assert np.all(np.abs(r["dist"][i, :c] - d64) <= 1e-5 * np.maximum(d64, 1e-30))
    assert oracle.recall(r["ids"], ex[0], ex[2], w.k).mean() >= (0.97 if dtype == "FP8E4M3" else 0.99)
    w, path = c2_small_index
    ix = U.Index(path)
    lo, hi = w.lo.copy(), w.hi.copy()
    lo[::7], hi[::7] = hi[::7] + 1, hi[::7]   # reversed: empty
    lo[3::11] = hi[3::11]                      # a single value
    lo[5::13], hi[5::13] = -10, -1             # below every attribute
    ex_ids, ex_d, ex_c = oracle.exact_knn(w.vectors, w.attrs, w.queries, lo, hi, w.k)
    tc = _np(ix.search(w.queries, lo, hi, w.k, strategy="pre",
                       params=U.Params.defaults(dtype=dt, rerank_mult=4, tc_scan=1)))
    assert np.array_equal(tc["count"], ex_c) and np.all(tc["status"] == 0), dtype
    if dtype != "FP8E4M3":
        fin = np.isfinite(ex_d)
        assert np.array_equal(tc["ids"], ex_ids), dtype
        assert np.array_equal(tc["dist"][fin].astype(np.float64), ex_d[fin]), dtype
    _valid(w, tc, lo, hi)
    assert (ex_c == 0).sum() >= len(lo) // 7


def test_c4_precision_shape_k10_k100(U, c4_small_index):
    """The precision shape (unit-normalised d = 96 mixture, ranges 1/10/50 %) at
    n = 20,000, auto-routed, at k = 10 and k = 100: BF16 and FP8 E4M3 storage with the
    FP32 re-rank of 4k candidates. Every returned distance is the float32 direct
    distance of its id (within 1e-5 of FP64); per range fraction, recall against the
    exact answer is at least 0.95 with FP32 storage and loses at most 0.03 (BF16) and
    0.06 (FP8) against it at the same parameters, and the rows routed to the
    pre-filter scan stay near exact."""
    w, path = c4_small_index
    ix = U.Index(path)
    X = w.vectors.astype(np.float64)
    ta, tb = w.n // 100, w.n // 2
    fr = np.unique(w.fractions)
    pre = oracle.OracleIndex(path).route(w.lo, w.hi, ta, tb)["strategy"] == 0
    assert 0 < pre.sum() < len(pre)
    report = {}
    for k in (10, 100):
        ex_ids, _, ex_c = oracle.exact_knn(w.vectors, w.attrs, w.queries, w.lo, w.hi, k)
        rec = {}
        for dtype in (U.FP32, U.BF16, U.FP8E4M3):
            p = U.Params.defaults(dtype=dtype, rerank_mult=4, tau_a=ta, tau_b=tb, m=32, ef_post=max(256, 2 * k),
                                  cand_cap=CAND, visited_cap=2048)
            r = _np(ix.search(w.queries, w.lo, w.hi, k, ef=max(128, 2 * k), strategy="auto", params=p))
            _valid(w, r, w.lo, w.hi)
            for i in range(len(w.lo)):
                c = r["count"][i]
                ids = r["ids"][i, :c]
                d64 = ((X[ids] - w.queries[i].astype(np.float64)) ** 2).sum(1)
                assert np.all(np.abs(r["dist"][i, :c] - d64) <= 1e-5 * np.maximum(d64, 1e-30)), (k, dtype)
            rr = oracle.recall(r["ids"], ex_ids, ex_c, k)
            rec[dtype] = {float(f): float(rr[w.fractions == f].mean()) for f in fr}
            rec[dtype]["pre"] = float(rr[pre].mean())
        report[k] = rec
        for f in fr:
            f = float(f)
            assert rec[U.FP32][f] >= 0.95, (k, f, rec)  # the recall@k target of every range fraction
            assert rec[U.BF16][f] >= rec[U.FP32][f] - 0.03, (k, f, rec)
            assert rec[U.FP8E4M3][f] >= rec[U.FP32][f] - 0.06, (k, f, rec)
        assert rec[U.BF16]["pre"] >= 0.98 and rec[U.FP8E4M3]["pre"] >= 0.95, (k, rec)
    print("c4-shape recall by k, dtype, fraction:", json.dumps({str(k): {str(d): v for d, v in r_.items()}
                                                                 for k, r_ in report.items()}))


@pytest.mark.parametrize("tc", [0, 1])
@pytest.mark.parametrize("dtype", ["BF16", "FP8E4M3"])
def test_wide_rerank_reduced_precision(U, tmp_path, dtype, tc):
    """BF16 and FP8 storage with twice the usual FP32 re-rank (8k candidates, a shape
    the autotuner tries), on either pre-filter scan, auto-routed: every row in range,
    every returned distance the FP32 direct distance of its id, and recall against the
    exact answer (Definition 1) at least 0.95."""
    import hsig_build
    from workloads import make_workload
    w = make_workload("c2", seed=5, n=20000, nq=600)
    path = str(tmp_path / "rr8.idx")
    hsig_build.build_index(w.vectors, w.attrs, path, w.S, w.M, 60, seed=5)
    ix = U.Index(path, device=0)
    ex_ids, _, ex_c = oracle.exact_knn(w.vectors, w.attrs, w.queries, w.lo, w.hi, w.k)
    X = w.vectors.astype(np.float64)
    p = U.Params.defaults(dtype=getattr(U, dtype), rerank_mult=8, tc_scan=tc, tau_a=w.n // 50, tau_b=w.n // 2)
    r = _np(ix.search(w.queries, w.lo, w.hi, w.k, ef=64, strategy="auto", params=p))
    _valid(w, r, w.lo, w.hi)
    for i in range(len(w.lo)):
        c = r["count"][i]
        ids = r["ids"][i, :c]
        d64 = ((X[ids] - w.queries[i].astype(np.float64)) ** 2).sum(1)
        assert np.all(np.abs(r["dist"][i, :c] - d64) <= 1e-5 * np.maximum(d64, 1e-30))
    assert oracle.recall(r["ids"], ex_ids, ex_c, w.k).mean() >= 0.95
    ix.close()
