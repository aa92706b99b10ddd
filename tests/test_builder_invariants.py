"""Structural invariants of the HSIG the host builder writes (Section 4.1, 4.3)."""
import numpy as np

import hsig_build


def _check(w, path):
    ix = hsig_build.read_index(path, verify=True)
    n, S, M = ix["n"], ix["S"], ix["M"]
    A = ix["attr"]
    assert np.array_equal(ix["vectors"], w.vectors) and np.array_equal(A, w.attrs)
    b = ix["seg_bounds"]
    seg = np.searchsorted(b[1:S], A, side="right")
    assert np.array_equal(np.bincount(seg, minlength=S), ix["seg_count"])
    # equi-depth bounds from all attributes (reading of Section 3.1)
    order = np.lexsort((np.arange(n), A))
    assert np.array_equal(ix["sorted_ids"], order)
    assert list(b[1:S]) == [int(A[order[j * n // S]]) for j in range(1, S)]
    # skip list: the level-0 chain is the attribute order; level-l chains hold level >= l
    lv = ix["level"]
    assert ix["skip_head"][0] == order[0]
    nxt = ix["skip_next0"]
    assert np.array_equal(nxt[order[:-1]], order[1:]) and nxt[order[-1]] == -1
    ub = ix["upper_base"]
    for l in range(1, ix["max_level"] + 1):
        chain = order[lv[order] >= l]
        assert ix["skip_head"][l] == chain[0]
        got = ix["skip_nextU"][ub[chain] + l - 1]
        assert np.array_equal(got[:-1], chain[1:]) and got[-1] == -1
    # upper rows are laid out by id
    up = np.flatnonzero(lv > 0)
    assert np.array_equal(ub[up], np.concatenate([[0], np.cumsum(lv[up])[:-1]]))
    assert ix["n_upper"] == lv.sum()
    # entry point: first object on the top layer
    assert lv[ix["entry_global"]] == ix["max_level"] == lv.max()
    assert ix["entry_global"] == np.flatnonzero(lv == lv.max())[0]
    # chunks: segment-pure, <= M, no duplicates/self loops, sorted by (distance, id), -1 padded
    X = w.vectors.astype(np.float64)
    for name, owners_of in (("adj0", np.arange(n)), ("adjU", None)):
        adj = ix[name]
        if name == "adjU":
            if ix["n_upper"] == 0:
                continue
            owners_of = np.repeat(up, lv[up])
            layer = np.concatenate([np.arange(1, v + 1) for v in lv[up]])
        for r in range(0, adj.shape[0], max(1, adj.shape[0] // 2000)):
            v = owners_of[r]
            for j in range(S):
                ch = adj[r, j]
                c = int((ch >= 0).sum())
                assert np.all(ch[:c] >= 0) and np.all(ch[c:] == -1)
                ids = ch[:c]
                assert np.all(seg[ids] == j) and v not in ids and len(set(ids.tolist())) == c
                if name == "adjU":
                    assert np.all(lv[ids] >= layer[r])
                dd = ((X[ids] - X[v]) ** 2).sum(1)
                keys = list(zip(dd.tolist(), ids.tolist()))
                assert keys == sorted(keys)
    # global-edge bitmaps: at most M bits, only on filled slots (Algorithm 5)
    for gname, aname in (("gmask0", "adj0"), ("gmaskU", "adjU")):
        if gname == "gmaskU" and ix["n_upper"] == 0:
            continue
        bits = np.unpackbits(ix[gname].view(np.uint8), axis=1, bitorder="little")
        assert bits.sum(1).max() <= M
        assert not bits[:, S * M:].any()
        filled = (ix[aname].reshape(ix[aname].shape[0], S * M) >= 0)
        assert not (bits[:, :S * M].astype(bool) & ~filled).any()
    return ix


def test_builder_invariants_c1(c1_index):
    w, path = c1_index
    ix = _check(w, path)
    # levels: P(level >= 1) = 1/M for mL = 1/ln M
    frac = (ix["level"] >= 1).mean()
    assert abs(frac - 1 / ix["M"]) < 0.02


def test_builder_invariants_c2_small(c2_small_index):
    w, path = c2_small_index
    _check(w, path)


def test_builder_is_deterministic(tmp_path):
    from workloads import make_workload
    w = make_workload("c1", n=3000, nq=4)
    p1, p2 = str(tmp_path / "a.idx"), str(tmp_path / "b.idx")
    hsig_build.build_index(w.vectors, w.attrs, p1, w.S, w.M, 40, seed=3, threads=1)
    hsig_build.build_index(w.vectors, w.attrs, p2, w.S, w.M, 40, seed=3, threads=4)
    with open(p1, "rb") as f1, open(p2, "rb") as f2:
        assert f1.read() == f2.read()


def test_inclusiveness_of_contiguous_segment_combinations(tmp_path):
    """Section 5.4's inclusiveness metric on the c1 shape (eight equal segments):
    for 1, 2, 4, 6 and 8 contiguous segments, an HNSW is built on those segments'
    objects alone (the builder with one segment), and the share of its layer-0 edges
    that the HSIG also holds, within the same segments, is averaged over several
    placements of the combination. The paper reports above 80 % for every size."""
    from workloads import make_workload
    w = make_workload("c1", seed=7)
    path = str(tmp_path / "hsig.idx")
    hsig_build.build_index(w.vectors, w.attrs, path, w.S, w.M, w.efc, seed=7)
    ix = hsig_build.read_index(path)
    n, S, M = ix["n"], ix["S"], ix["M"]
    seg = np.searchsorted(ix["seg_bounds"][1:S], w.attrs, side="right")
    adj = np.asarray(ix["adj0"]).reshape(n, S * M)
    hsig_edges = {(v, int(u)) for v in range(n) for u in adj[v] if u >= 0}
    report = {}
    for c, starts in ((1, (0, 3, 7)), (2, (0, 3, 6)), (4, (0, 4)), (6, (0, 2)), (8, (0,))):
        vals = []
        for s0 in starts:
            members = np.flatnonzero((seg >= s0) & (seg < s0 + c))
            sub = str(tmp_path / f"hnsw_{c}_{s0}.idx")
            hsig_build.build_index(w.vectors[members], w.attrs[members], sub, 1, M, w.efc, seed=7)
            h = hsig_build.read_index(sub)
            hadj = np.asarray(h["adj0"]).reshape(len(members), M)
            vv, ss = np.nonzero(hadj >= 0)
            edges = list(zip(members[vv].tolist(), members[hadj[vv, ss]].tolist()))
            vals.append(sum(e in hsig_edges for e in edges) / len(edges))
        report[c] = float(np.mean(vals))
    print("inclusiveness by contiguous segments:", report)
    assert all(v > 0.8 for v in report.values()), report
