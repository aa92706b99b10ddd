"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test names the passage it checks. None of them re-types the oracle's own
formulas: they use brute force in plain Python, library routines (numpy sort and
searchsorted, scipy graph components), hand-traced examples and properties
(Lemma 1 / Theorem 1) that a wrong oracle would violate.
"""
import itertools
import json
import os

import numpy as np
import pytest

import oracle
from index_writer import tiny_index_sections, write_index

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- O1 (Definition 1)

def _py_bruteforce(X, A, q, lo, hi, k):
    """Definition 1 by hand: integer data, exact Python integers."""
    R = [i for i in range(len(A)) if lo <= A[i] <= hi]
    d = [(sum((int(q[t]) - int(X[i][t])) ** 2 for t in range(len(q))), i) for i in R]
    d.sort()
    return d[:k]


def test_exact_knn_equals_python_bruteforce():
    rng = np.random.default_rng(5)
    n, d = 60, 3
    X = rng.integers(0, 6, size=(n, d)).astype(np.float32)  # many distance ties
    A = rng.integers(0, 20, size=n).astype(np.int64)
    Q = rng.integers(0, 6, size=(25, d)).astype(np.float32)
    lo = rng.integers(-2, 15, size=25)
    hi = lo + rng.integers(0, 10, size=25)
    for k in (1, 4, 9):
        ids, dist, cnt = oracle.exact_knn(X, A, Q, lo, hi, k)
        for i in range(25):
            ref = _py_bruteforce(X, A, Q[i], lo[i], hi[i], k)
            assert cnt[i] == len(ref)
            assert list(ids[i, :cnt[i]]) == [r[1] for r in ref]
            assert list(dist[i, :cnt[i]]) == [float(r[0]) for r in ref]
            assert np.all(ids[i, cnt[i]:] == -1) and np.all(np.isinf(dist[i, cnt[i]:]))


def test_exact_knn_short_and_empty_ranges():
    """|R| < k returns all of R (Definition 1); an empty range returns nothing."""
    X = np.arange(10, dtype=np.float32).reshape(10, 1)
    A = np.arange(10, dtype=np.int64) * 10
    Q = np.array([[4.2], [4.2], [4.2], [0.0]], np.float32)
    lo = np.array([30, 95, 50, 0])
    hi = np.array([50, 99, 40, 1000])
    ids, dist, cnt = oracle.exact_knn(X, A, Q, lo, hi, 5)
    assert list(cnt) == [3, 0, 0, 5]
    assert list(ids[0, :3]) == [4, 5, 3]
    assert list(ids[3]) == [0, 1, 2, 3, 4]
    assert np.all(ids[1] == -1) and np.all(ids[2] == -1)


def test_exact_knn_self_query_is_first():
    rng = np.random.default_rng(9)
    X = rng.standard_normal((300, 8)).astype(np.float32)
    A = rng.permutation(300).astype(np.int64)
    v = np.arange(0, 300, 17)
    ids, dist, cnt = oracle.exact_knn(X, A, X[v], A[v] - 5, A[v] + 5, 3)
    assert np.all(ids[:, 0] == v) and np.all(dist[:, 0] == 0.0)
    assert np.all(dist[:, 1] > 0.0)


def test_theorem1_sig_knng_inclusive():
    """Lemma 1 / Theorem 1 (Section 3.2): with per-segment kNN chunks (SIG-kNNG),
    the kNN graph of every union of segments is a sub-graph. Built by brute force
    with O1 on a small input; a wrong range filter or ranking breaks it."""
    rng = np.random.default_rng(11)
    n, d, S, k = 64, 4, 4, 3
    X = rng.standard_normal((n, d)).astype(np.float32)
    A = rng.permutation(n).astype(np.int64)
    seg_lo = [j * n // S for j in range(S)]
    seg_hi = [(j + 1) * n // S - 1 for j in range(S)]
    # chunk j of v = kNN(v, D_j \ {v}); ask k+1 and drop v itself (distance 0, unique)
    chunks = {}
    for j in range(S):
        ids, _, cnt = oracle.exact_knn(X, A, X, np.full(n, seg_lo[j]), np.full(n, seg_hi[j]), k + 1)
        for v in range(n):
            chunks[(v, j)] = [int(o) for o in ids[v, :cnt[v]] if o != v][:k]
    sig = {v: set(itertools.chain.from_iterable(chunks[(v, j)] for j in range(S))) for v in range(n)}
    for a in range(S):
        for b in range(a, S):
            lo, hi = seg_lo[a], seg_hi[b]
            members = [v for v in range(n) if lo <= A[v] <= hi]
            ids, _, cnt = oracle.exact_knn(X, A, X[members], np.full(len(members), lo),
                                           np.full(len(members), hi), k + 1)
            for r, v in enumerate(members):
                knn = [int(o) for o in ids[r, :cnt[r]] if o != v][:k]
                assert all(lo <= A[o] <= hi for o in knn)
                assert set(knn) <= sig[v], (v, a, b)


# ---------------------------------------------------------------- Eq. 1

def test_recall_formula():
    ex = np.array([[1, 2, 3], [7, -1, -1], [-1, -1, -1]])
    cnt = np.array([3, 1, 0])
    fo = np.array([[3, 9, 1], [8, 7, -1], [-1, -1, -1]])
    r = oracle.recall(fo, ex, cnt, 3)
    assert r[0] == pytest.approx(2 / 3) and r[1] == 1.0 and r[2] == 1.0


# ---------------------------------------------------------------- hand-traced (Alg. 1, 7)

@pytest.fixture(scope="module")
def tiny(tmp_path_factory):
    with open(os.path.join(GOLDEN, "tiny_line_graph.json")) as f:
        g = json.load(f)
    path = str(tmp_path_factory.mktemp("tiny") / "tiny.idx")
    write_index(path, tiny_index_sections(g))
    return g, path


def test_golden_tiny_line_graph(tiny):
    g, path = tiny
    oi = oracle.OracleIndex(path)
    for case in g["cases"]:
        r = oi.search(np.array([case["q"]], np.float32), [case["lo"]], [case["hi"]], case["k"],
                      ef=case["ef"], m=case["m"], ef_post=case["ef"], strategy=case["strategy"])
        want = case["expect_ids"]
        assert list(r["ids"][0]) == want, case["name"]
        for got, exp in zip(r["dist"][0], case["expect_dist"]):
            if exp is None:
                assert np.isinf(got)
            else:
                assert got == pytest.approx(exp, rel=1e-6, abs=1e-6), case["name"]
        assert r["n_exp"][0] == case["expect_n_exp"], case["name"]
        assert r["n_dist"][0] == case["expect_n_dist"], case["name"]


def test_corrupt_index_is_rejected(tiny, tmp_path):
    g, _ = tiny
    path = str(tmp_path / "bad.idx")
    write_index(path, tiny_index_sections(g), corrupt_section="adj0")
    with pytest.raises(RuntimeError):
        oracle.OracleIndex(path)


# ---------------------------------------------------------------- routing (Section 4.2)

def test_paper_segmentation_example(tmp_path):
    """Section 3.2 example: attributes 1..8 in two segments [1,5) and [5,8]."""
    with open(os.path.join(GOLDEN, "segmentation_example.json")) as f:
        g = json.load(f)
    import hsig_build
    X = np.arange(8, dtype=np.float32).reshape(8, 1)
    A = np.array(g["attributes"], np.int64)
    path = str(tmp_path / "seg.idx")
    hsig_build.build_index(X, A, path, S=g["S"], M=2, efc=4, seed=1)
    ix = hsig_build.read_index(path)
    assert list(ix["seg_bounds"][1:-1]) == g["expect_inner_bounds"]
    oi = oracle.OracleIndex(path)
    lo = np.array([c[0] for c in g["mask_cases"]])
    hi = np.array([c[1] for c in g["mask_cases"]])
    r = oi.route(lo, hi)
    assert list(r["mask"]) == [c[2] for c in g["mask_cases"]]


def test_route_bounds_masks_strategies(c1_index):
    w, path = c1_index
    import hsig_build
    ix = hsig_build.read_index(path)
    oi = oracle.OracleIndex(path)
    rng = np.random.default_rng(3)
    sa = np.sort(w.attrs)
    lo = np.concatenate([rng.integers(-50, w.n + 50, 400), [0, 0, 5, -10, w.n - 1, 100]])
    hi = np.concatenate([lo[:400] + rng.integers(-3, w.n // 2, 400), [w.n - 1, 99, 4, -1, w.n + 5, 199]])
    tau_a, tau_b = 100, 5000
    r = oi.route(lo, hi, tau_a, tau_b)
    pa = np.searchsorted(sa, lo, side="left")
    pb = np.maximum(np.searchsorted(sa, hi, side="right"), pa)
    assert np.array_equal(r["pa"], pa) and np.array_equal(r["pb"], pb)
    Y = pb - pa
    want = np.where(Y <= tau_a, 0, np.where(Y >= tau_b, 2, 1))
    assert np.array_equal(r["strategy"], want)
    b = ix["seg_bounds"]
    S = ix["S"]
    seg_of = np.searchsorted(b[1:S], w.attrs, side="right")
    for i in range(len(lo)):
        m = int(r["mask"][i])
        inr = (w.attrs >= lo[i]) & (w.attrs <= hi[i])
        # every in-range object's segment is marked
        for j in np.unique(seg_of[inr]):
            assert (m >> int(j)) & 1
        # every marked segment's interval overlaps [lo, hi] and holds objects
        for j in range(S):
            if (m >> j) & 1:
                lo_j = -np.inf if j == 0 else b[j]
                hi_j = np.inf if j == S - 1 else b[j + 1] - 1
                assert max(lo_j, lo[i]) <= min(hi_j, hi[i])
                assert (seg_of == j).any()
        # skip-list descent lands on the first object with attribute >= lo
        first = int(r["first"][i])
        n_below = int(np.searchsorted(sa, lo[i], side="left"))
        assert first == (int(ix["sorted_ids"][n_below]) if n_below < w.n else -1)


def test_router_thresholds_at_exact_counts(c1_index):
    """Y <= tau_A -> A, Y >= tau_B -> B, otherwise C, at the boundary counts (c1's
    attribute is a permutation, so a width-w range holds exactly w objects)."""
    w, path = c1_index
    oi = oracle.OracleIndex(path)
    tau_a, tau_b = 100, 5000
    widths = np.array([0, 1, 99, 100, 101, 4999, 5000, 5001, w.n])
    lo = np.full(len(widths), 0)
    hi = widths - 1
    r = oi.route(lo, hi, tau_a, tau_b)
    assert list(r["pb"] - r["pa"]) == list(widths)
    assert list(r["strategy"]) == [0, 0, 0, 0, 1, 1, 2, 2, 2]


# ---------------------------------------------------------------- strategies vs O1

def test_prefilter_equals_exact(c1_index):
    """Strategy A is exact (Section 4.2): equal to Definition 1 id for id."""
    w, path = c1_index
    oi = oracle.OracleIndex(path)
    ex = oracle.exact_knn(w.vectors, w.attrs, w.queries, w.lo, w.hi, w.k)
    r = oi.search(w.queries, w.lo, w.hi, w.k, strategy="pre")
    assert np.array_equal(r["ids"], ex[0]) and np.array_equal(r["count"], ex[2])
    assert np.array_equal(r["dist"], ex[1])


def _flat_copy(path, out_path):
    """The same layer-0 graph with the upper layers dropped, so that the search
    starts at the stored entry point on layer 0."""
    import hsig_build
    ix = hsig_build.read_index(path)
    n, S, M, W = ix["n"], ix["S"], ix["M"], ix["W"]
    meta = np.array(ix["meta"], np.int64)
    meta[4] = 0
    meta[6] = 0
    sec = {k: np.array(ix[k]) for k in ("vectors", "attr", "seg_bounds", "seg_count", "entry_seg",
                                         "sorted_ids", "skip_next0", "adj0", "gmask0")}
    sec.update(meta=meta, level=np.zeros(n, np.int32), upper_base=np.full(n, -1, np.int32),
               skip_head=np.array([ix["sorted_ids"][0]], np.int32), skip_nextU=np.full(1, -1, np.int32),
               adjU=np.full((1, S, M), -1, np.int32), gmaskU=np.zeros((1, W), np.uint32))
    write_index(out_path, sec)
    return ix


def _closure(n, src, dst, start):
    from scipy.sparse import coo_matrix
    from scipy.sparse.csgraph import breadth_first_order
    g = coo_matrix((np.ones(len(src)), (src, dst)), shape=(n, n)).tocsr()
    return breadth_first_order(g, start, directed=True, return_predecessors=False)


def _topk_fp64(X, q, ids, k):
    d = ((X[ids].astype(np.float64) - q.astype(np.float64)) ** 2).sum(1)
    o = np.lexsort((ids, d))[:k]
    return ids[o]


def test_hybrid_unbounded_beam_is_exact(c1_index, tmp_path):
    """With ef above |R| the ann never fills, Algorithm 7 never breaks and expands
    every node reachable from the entry point over the selected chunk slots (S2).
    The result must then be the exact top-k of the in-range part of that closure
    (scipy BFS + numpy sort)."""
    w, path = c1_index
    flat = str(tmp_path / "flat.idx")
    ix = _flat_copy(path, flat)
    n, S, M = ix["n"], ix["S"], ix["M"]
    oi = oracle.OracleIndex(flat)
    sel = np.flatnonzero(w.fractions <= 0.10)[:40]
    Q, lo, hi = w.queries[sel], w.lo[sel], w.hi[sel]
    m = 16
    r = oi.search(Q, lo, hi, w.k, ef=n, m=m, strategy="hybrid")
    rt = oi.route(lo, hi)
    ep = ix["entry_global"]
    nonempty = 0
    for i in range(len(sel)):
        mask = int(rt["mask"][i])
        segs = [j for j in range(S) if (mask >> j) & 1]
        per = min(M, -(-m // len(segs)))
        src, dst = [], []
        for j in segs:
            ch = ix["adj0"][:, j, :per]
            vv, ss = np.nonzero(ch >= 0)
            src.append(vv)
            dst.append(ch[vv, ss])
        reach = _closure(n, np.concatenate(src), np.concatenate(dst), ep)
        inr = reach[(w.attrs[reach] >= lo[i]) & (w.attrs[reach] <= hi[i])]
        want = _topk_fp64(w.vectors, Q[i], inr, w.k)
        nonempty += len(want) > 0
        assert int(r["count"][i]) == len(want)
        assert np.array_equal(r["ids"][i, :len(want)], want), i
    assert nonempty >= 30


def test_hybrid_s1_unbounded_beam_is_exact(c1_index, tmp_path):
    """Selection S1 (Section 4.2's first strategy): every neighbour in the intersected
    chunks, ordered by distance to the expanded object, the first m. With ef above
    |R| the result must be the exact top-k of the in-range part of the closure over
    those edges, computed here independently: numpy FP64 owner distances, lexsort by
    (distance, id), the first m per object, scipy BFS. The S1 edges must also differ
    from the S2 edges of the same m for some query (the pin is not vacuous)."""
    w, path = c1_index
    flat = str(tmp_path / "flat.idx")
    ix = _flat_copy(path, flat)
    n, S, M = ix["n"], ix["S"], ix["M"]
    adj = np.asarray(ix["adj0"]).reshape(n, S * M)
    X = w.vectors.astype(np.float64)
    safe = np.where(adj >= 0, adj, 0)
    dv = ((X[safe] - X[:, None, :]) ** 2).sum(-1)  # owner distance of every slot
    oi = oracle.OracleIndex(flat)
    sel = np.flatnonzero(w.fractions <= 0.10)[:24]
    Q, lo, hi = w.queries[sel], w.lo[sel], w.hi[sel]
    m = 8
    r = oi.search(Q, lo, hi, w.k, ef=n, m=m, strategy="hybrid", selection=1)
    rt = oi.route(lo, hi)
    ep = ix["entry_global"]
    nonempty = differs = 0
    slot_seg = np.repeat(np.arange(S), M)
    for i in range(len(sel)):
        mask = int(rt["mask"][i])
        ok = (adj >= 0) & (((mask >> slot_seg) & 1) == 1)[None, :]
        d = np.where(ok, dv, np.inf)
        ids = np.where(ok, adj, np.iinfo(np.int32).max)
        order = np.lexsort((ids, d), axis=-1)[:, :m]
        pick = np.take_along_axis(ok, order, axis=1)
        vv = np.repeat(np.arange(n), m).reshape(n, m)[pick]
        uu = np.take_along_axis(adj, order, axis=1)[pick]
        reach = _closure(n, vv, uu, ep)
        inr = reach[(w.attrs[reach] >= lo[i]) & (w.attrs[reach] <= hi[i])]
        want = _topk_fp64(w.vectors, Q[i], inr, w.k)
        nonempty += len(want) > 0
        assert int(r["count"][i]) == len(want), i
        assert np.array_equal(r["ids"][i, :len(want)], want), i
        segs = [j for j in range(S) if (mask >> j) & 1]
        per = min(M, -(-m // len(segs)))
        ch = adj.reshape(n, S, M)[:, segs, :per].reshape(n, -1)
        v2, t2 = np.nonzero(ch >= 0)
        differs += set(zip(v2.tolist(), ch[v2, t2].tolist())) != set(zip(vv.tolist(), uu.tolist()))
    assert nonempty >= 16
    assert differs >= 1


def test_s1_with_every_slot_equals_s2(c1_index):
    """With m >= S'M both selections take every neighbour in the intersected chunks
    (S1 only orders them differently, and one expansion's neighbours give the same
    outcome in any order), so S1 and S2 must agree on ids, distances and counts."""
    w, path = c1_index
    oi = oracle.OracleIndex(path)
    m = 16 * 32
    a = oi.search(w.queries, w.lo, w.hi, w.k, ef=64, m=m, strategy="hybrid", selection=2)
    b = oi.search(w.queries, w.lo, w.hi, w.k, ef=64, m=m, strategy="hybrid", selection=1)
    for key in ("ids", "dist", "count", "n_dist", "n_exp"):
        assert np.array_equal(a[key], b[key]), key


def test_post_unbounded_beam_is_exact(c1_index, tmp_path):
    """Strategy B with ef_post >= n keeps every node reachable from the entry point
    over the bitmap-marked slots; after the range filter the result must be the
    exact top-k of the in-range part of that closure."""
    w, path = c1_index
    flat = str(tmp_path / "flat.idx")
    ix = _flat_copy(path, flat)
    n, S, M = ix["n"], ix["S"], ix["M"]
    bits = np.unpackbits(ix["gmask0"].view(np.uint8), axis=1, bitorder="little")[:, :S * M].astype(bool)
    adj = ix["adj0"].reshape(n, S * M)
    vv, pp = np.nonzero(bits & (adj >= 0))
    reach = _closure(n, vv, adj[vv, pp], ix["entry_global"])
    assert len(reach) > 0.9 * n
    oi = oracle.OracleIndex(flat)
    sel = np.arange(0, len(w.lo), 5)
    Q, lo, hi = w.queries[sel], w.lo[sel], w.hi[sel]
    r = oi.search(Q, lo, hi, w.k, ef=100, ef_post=n, strategy="post")
    for i in range(len(sel)):
        inr = reach[(w.attrs[reach] >= lo[i]) & (w.attrs[reach] <= hi[i])]
        want = _topk_fp64(w.vectors, Q[i], inr, w.k)
        assert np.array_equal(r["ids"][i, :len(want)], want) and int(r["count"][i]) == len(want)


def test_results_are_valid(c1_index):
    """Invariants of every strategy: ids in [lo, hi], sorted by (distance, id), no
    duplicates, padding after count (Definition 1)."""
    w, path = c1_index
    oi = oracle.OracleIndex(path)
    for st in ("pre", "hybrid", "post", "auto"):
        r = oi.search(w.queries, w.lo, w.hi, w.k, ef=40, strategy=st, tau_a=100, tau_b=5000)
        for i in range(len(w.lo)):
            c = int(r["count"][i])
            ids, dist = r["ids"][i, :c], r["dist"][i, :c]
            assert np.all((w.attrs[ids] >= w.lo[i]) & (w.attrs[ids] <= w.hi[i]))
            assert len(set(ids.tolist())) == c
            keys = list(zip(dist.tolist(), ids.tolist()))
            assert keys == sorted(keys)
            assert np.all(r["ids"][i, c:] == -1)
        if st in ("pre", "hybrid"):
            ex_cnt = np.minimum(w.k, np.array([((w.attrs >= a) & (w.attrs <= b)).sum() for a, b in zip(w.lo, w.hi)]))
            if st == "pre":
                assert np.array_equal(r["count"], ex_cnt)


def _conj(w, seed=11):
    from workloads import second_attribute
    fr = np.array([0.2, 0.5, 1.0])[np.arange(len(w.lo)) % 3]
    return second_attribute(w.n, fr, seed)


def test_conjunctive_exact_equals_bruteforce(c1_index):
    """O1 with a second attribute (lo <= A1 <= hi AND lo2 <= A2 <= hi2) against a
    numpy FP64 brute force with lexsort by (distance, id): ids equal, distances equal
    up to the rounding of a different summation order."""
    w, _ = c1_index
    a2, lo2, hi2 = _conj(w)
    ids, dist, cnt = oracle.exact_knn(w.vectors, w.attrs, w.queries, w.lo, w.hi, w.k, attr2=a2, lo2=lo2, hi2=hi2)
    X = w.vectors.astype(np.float64)
    for i in range(len(w.lo)):
        inr = np.flatnonzero((w.attrs >= w.lo[i]) & (w.attrs <= w.hi[i]) & (a2 >= lo2[i]) & (a2 <= hi2[i]))
        d = ((X[inr] - w.queries[i].astype(np.float64)) ** 2).sum(1)
        o = np.lexsort((inr, d))[:w.k]
        c = len(o)
        # same ids; FP64 sums in another order agree to rounding
        assert cnt[i] == c and np.array_equal(ids[i, :c], inr[o])
        assert np.allclose(dist[i, :c], d[o], rtol=1e-12, atol=0)
        assert np.all(ids[i, c:] == -1)


def test_conjunctive_pre_equals_exact(c1_index):
    """Strategy A with the conjunctive predicate equals O1 with it."""
    w, path = c1_index
    a2, lo2, hi2 = _conj(w)
    oi = oracle.OracleIndex(path)
    ex = oracle.exact_knn(w.vectors, w.attrs, w.queries, w.lo, w.hi, w.k, attr2=a2, lo2=lo2, hi2=hi2)
    r = oi.search(w.queries, w.lo, w.hi, w.k, strategy="pre", attr2=a2, lo2=lo2, hi2=hi2)
    assert np.array_equal(r["ids"], ex[0]) and np.array_equal(r["count"], ex[2])
    assert np.array_equal(r["dist"], ex[1])


def test_conjunctive_unbounded_beams_are_exact(c1_index, tmp_path):
    """With the beam above n, hybrid (S2 edges of the A1 mask) and post-filter (bitmap
    edges) reach their whole closure; the conjunctive result must be the exact top-k
    of the closure's objects satisfying both ranges (scipy BFS + numpy sort)."""
    w, path = c1_index
    flat = str(tmp_path / "flat.idx")
    ix = _flat_copy(path, flat)
    n, S, M = ix["n"], ix["S"], ix["M"]
    a2, lo2, hi2 = _conj(w)
    oi = oracle.OracleIndex(flat)
    sel = np.flatnonzero(w.fractions <= 0.10)[:30]
    Q, lo, hi, l2, h2 = w.queries[sel], w.lo[sel], w.hi[sel], lo2[sel], hi2[sel]
    m = 16
    rh = oi.search(Q, lo, hi, w.k, ef=n, m=m, strategy="hybrid", attr2=a2, lo2=l2, hi2=h2)
    rp = oi.search(Q, lo, hi, w.k, ef=100, ef_post=n, strategy="post", attr2=a2, lo2=l2, hi2=h2)
    rt = oi.route(lo, hi)
    ep = ix["entry_global"]
    bits = np.unpackbits(ix["gmask0"].view(np.uint8), axis=1, bitorder="little")[:, :S * M].astype(bool)
    adj = ix["adj0"].reshape(n, S * M)
    vv, pp = np.nonzero(bits & (adj >= 0))
    reach_b = _closure(n, vv, adj[vv, pp], ep)
    nonempty = 0
    for i in range(len(sel)):
        mask = int(rt["mask"][i])
        segs = [j for j in range(S) if (mask >> j) & 1]
        per = min(M, -(-m // len(segs)))
        src, dst = [], []
        for j in segs:
            ch = ix["adj0"][:, j, :per]
            v_, s_ = np.nonzero(ch >= 0)
            src.append(v_)
            dst.append(ch[v_, s_])
        for reach, r in ((_closure(n, np.concatenate(src), np.concatenate(dst), ep), rh), (reach_b, rp)):
            ok = (w.attrs[reach] >= lo[i]) & (w.attrs[reach] <= hi[i]) & (a2[reach] >= l2[i]) & (a2[reach] <= h2[i])
            want = _topk_fp64(w.vectors, Q[i], reach[ok], w.k)
            nonempty += len(want) > 0
            assert int(r["count"][i]) == len(want), i
            assert np.array_equal(r["ids"][i, :len(want)], want), i
    assert nonempty >= 30


def test_conjunctive_full_second_range_is_single_attribute(c1_index):
    """A second range that holds every object leaves every strategy's result, and its
    distance and expansion counts, as without the second attribute."""
    w, path = c1_index
    oi = oracle.OracleIndex(path)
    a2, _, _ = _conj(w)
    lo2 = np.full(len(w.lo), -1, np.int64)
    hi2 = np.full(len(w.lo), 10**6, np.int64)
    for st in ("pre", "hybrid", "post", "auto"):
        a = oi.search(w.queries, w.lo, w.hi, w.k, ef=40, strategy=st, tau_a=100, tau_b=5000)
        b = oi.search(w.queries, w.lo, w.hi, w.k, ef=40, strategy=st, tau_a=100, tau_b=5000,
                      attr2=a2, lo2=lo2, hi2=hi2)
        for key in ("ids", "dist", "count", "n_dist", "n_exp", "strategy"):
            assert np.array_equal(a[key], b[key]), (st, key)


# ---------------------------------------------------------------- hierarchical descent (Algorithm 2)

@pytest.fixture(scope="module")
def layered(tmp_path_factory):
    from index_writer import layered_index_sections
    with open(os.path.join(GOLDEN, "layered_line_graph.json")) as f:
        g = json.load(f)
    path = str(tmp_path_factory.mktemp("layered") / "layered.idx")
    write_index(path, layered_index_sections(g))
    return g, path


def test_golden_layered_graph_search(layered):
    """Hand-traced searches on a three-layer index: Strategy C's upper layers take
    'lies in an intersected segment' as ann test and keep their entry point while ann
    stays empty; Strategy B's upper layers follow bitmap-marked slots only; both
    descend from the global entry point (Algorithm 2). Ids, distances, expansion and
    distance counts and the entry point of every layer are the traced ones."""
    g, path = layered
    oi = oracle.OracleIndex(path)
    assert oi.max_level == 2
    for case in g["cases"]:
        r = oi.search(np.array([case["q"]], np.float32), [case["lo"]], [case["hi"]], case["k"],
                      ef=case["ef"], m=case["m"], ef_post=case["ef"], strategy=case["strategy"], trace=True)
        assert list(r["ids"][0]) == case["expect_ids"], case["name"]
        for got, exp in zip(r["dist"][0], case["expect_dist"]):
            if exp is None:
                assert np.isinf(got), case["name"]
            else:
                assert got == exp, case["name"]  # exact: q = 9.5 and integer coordinates
        assert r["n_exp"][0] == case["expect_n_exp"], case["name"]
        assert r["n_dist"][0] == case["expect_n_dist"], case["name"]
        assert list(r["eps"][0]) == case["expect_eps"], case["name"]


def test_golden_layered_graph_route(layered):
    """Range bounds, masks and the skip-list descent through levels 2, 1 and 0 of the
    same index, against the traced values."""
    g, path = layered
    oi = oracle.OracleIndex(path)
    rc = g["route_cases"]
    r = oi.route(np.array([c["lo"] for c in rc]), np.array([c["hi"] for c in rc]))
    for i, c in enumerate(rc):
        assert int(r["mask"][i]) == c["mask"], c
        assert int(r["first"][i]) == c["first"], c
        assert (int(r["pa"][i]), int(r["pb"][i])) == (c["pa"], c["pb"]), c


def _upper_row(ix, v, l):
    return int(ix["upper_base"][v]) + l - 1


def _greedy_post_layer(ix, X, q, ep, l):
    """Algorithm 1 at ann size 1 is the greedy walk: move to the nearest of the current
    node and its bitmap-marked neighbours on layer l until the current node is the
    nearest (keys (squared distance, id), FP64)."""
    S, M = ix["S"], ix["M"]
    key = lambda v: (float(((X[v] - q) ** 2).sum()), int(v))
    cur = ep
    while True:
        row = _upper_row(ix, cur, l)
        adj = ix["adjU"][row].reshape(S * M)
        bits = np.unpackbits(ix["gmaskU"][row].view(np.uint8), bitorder="little")[:S * M].astype(bool)
        nb = [int(v) for v in adj[bits & (adj >= 0)]]
        best = min([key(cur)] + [key(v) for v in nb])
        if best[1] == cur:
            return cur
        cur = best[1]


def _frontier_hybrid_layer(ix, X, q, ep, l, mask, m, seg_of):
    """Algorithm 7 at ann size 1 on layer l, written as a best-first search with a
    threshold: the threshold is the best key seen among objects of intersected
    segments (none at first); an unseen selected neighbour joins the frontier when no
    threshold exists yet or its key is below it; the search stops when the frontier's
    nearest object is above the threshold. Selection S2: the first ceil(m / S') slots
    of each intersected chunk. Returns the object holding the threshold, or ep."""
    import heapq
    S, M = ix["S"], ix["M"]
    segs = [j for j in range(S) if (mask >> j) & 1]
    per = min(M, -(-m // len(segs)))
    key = lambda v: (float(((X[v] - q) ** 2).sum()), int(v))
    passes = lambda v: (mask >> int(seg_of[v])) & 1
    best = key(ep) if passes(ep) else None
    frontier, seen = [key(ep)], {ep}
    while frontier:
        o = heapq.heappop(frontier)
        if best is not None and best < o:
            break
        adj = ix["adjU"][_upper_row(ix, o[1], l)]
        for j in segs:
            for v in adj[j, :per]:
                v = int(v)
                if v < 0:
                    break
                if v in seen:
                    continue
                seen.add(v)
                kv = key(v)
                if best is None or kv < best:
                    heapq.heappush(frontier, kv)
                    if passes(v):
                        best = kv
    return ep if best is None else best[1]


def test_upper_layer_descent_matches_independent_restatement(c1_index):
    """The entry point of every layer of the oracle's hierarchical descent (Algorithm 2)
    equals an independent restatement: Strategy B as the greedy walk over bitmap
    slots, Strategy C as a threshold best-first search whose threshold comes from
    objects of intersected segments. Both start at the global entry point. The c1
    ranges cover parts of segments, so the segment test and the exact range test pick
    different entry points for many queries (checked, so the pin is not vacuous)."""
    import hsig_build
    w, path = c1_index
    ix = hsig_build.read_index(path)
    L = ix["max_level"]
    assert L >= 2
    S = ix["S"]
    seg_of = np.searchsorted(ix["seg_bounds"][1:S], w.attrs, side="right")
    X = w.vectors.astype(np.float64)
    oi = oracle.OracleIndex(path)
    m = 16
    sel = np.arange(0, len(w.lo), 2)
    Q, lo, hi = w.queries[sel], w.lo[sel], w.hi[sel]
    rc = oi.search(Q, lo, hi, w.k, ef=40, m=m, strategy="hybrid", trace=True)
    rb = oi.search(Q, lo, hi, w.k, ef=40, ef_post=40, strategy="post", trace=True)
    masks = oi.route(lo, hi)["mask"]
    inrange = lambda v, i: lo[i] <= w.attrs[v] <= hi[i]
    differs = 0
    for i in range(len(sel)):
        q = Q[i].astype(np.float64)
        ep_b = ep_c = ix["entry_global"]
        for l in range(L, 0, -1):
            assert rb["eps"][i, l] == ep_b, (i, l)
            assert rc["eps"][i, l] == ep_c, (i, l)
            ep_b = _greedy_post_layer(ix, X, q, ep_b, l)
            nxt = _frontier_hybrid_layer(ix, X, q, ep_c, l, int(masks[i]), m, seg_of)
            differs += int(nxt != ep_c and not inrange(nxt, i))
            ep_c = nxt
        assert rb["eps"][i, 0] == ep_b, i
        assert rc["eps"][i, 0] == ep_c, i
    # upper-layer entry points outside [lo, hi] but inside an intersected segment occur
    assert differs >= 10


def test_single_segment_full_range_post_equals_hybrid(c1_index, tmp_path):
    """With one segment, every chunk slot marked as a global edge and a range holding
    every object, Strategy C (S2 with m = M: every slot; the ann test always passes on
    every layer) and Strategy B (every slot is bitmap-marked; the filter keeps all)
    run the same Algorithm 2 over the same multi-layer graph. Ids, distances, counts,
    distance and expansion counts and the entry point of every layer must agree."""
    import hsig_build
    w, _ = c1_index
    path = str(tmp_path / "s1.idx")
    hsig_build.build_index(w.vectors, w.attrs, path, 1, 16, 60, seed=3)
    ix = hsig_build.read_index(path)
    assert ix["S"] == 1 and ix["max_level"] >= 2
    sec = {k: np.array(ix[k]) for k in ix if isinstance(ix[k], np.ndarray)}
    M, W = ix["M"], ix["W"]
    for a, g in (("adj0", "gmask0"), ("adjU", "gmaskU")):
        filled = (sec[a].reshape(sec[a].shape[0], M) >= 0)
        bits = np.zeros((filled.shape[0], W * 32), bool)
        bits[:, :M] = filled
        sec[g] = np.packbits(bits, axis=1, bitorder="little").view(np.uint32).reshape(-1, W)
    full = str(tmp_path / "s1_full_bitmap.idx")
    write_index(full, sec)
    oi = oracle.OracleIndex(full)
    lo = np.full(len(w.lo), w.attrs.min())
    hi = np.full(len(w.lo), w.attrs.max())
    for ef in (1, 10, 64):
        c = oi.search(w.queries, lo, hi, w.k, ef=ef, m=M, strategy="hybrid", trace=True)
        b = oi.search(w.queries, lo, hi, w.k, ef=ef, ef_post=ef, strategy="post", trace=True)
        for key in ("ids", "dist", "count", "n_dist", "n_exp", "eps"):
            assert np.array_equal(c[key], b[key]), (ef, key)
    assert np.all(c["eps"][:, ix["max_level"]] == ix["entry_global"])
