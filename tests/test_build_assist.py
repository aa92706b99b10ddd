"""Host side of GPU-assisted construction, without a GPU: the builder hands batches
of 64 or more nodes to a proposal callback, describes the graph through
unify_build_view_t (layout checked against include/unify.h), lists exactly the
chunks changed since the previous call (here: every non-empty chunk, on the first
call), and turns a callback error into a build error."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

import hsig_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


class View(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("d", ctypes.c_int), ("S", ctypes.c_int), ("M", ctypes.c_int),
                ("efc", ctypes.c_int), ("X", ctypes.c_void_p), ("level", ctypes.c_void_p),
                ("row0", ctypes.c_void_p), ("nrows", ctypes.c_int64), ("adj", ctypes.c_void_p),
                ("adjd", ctypes.c_void_p), ("cnt", ctypes.c_void_p), ("entry_seg", ctypes.c_void_p), ("top_seg", ctypes.c_void_p),
                ("dirty", ctypes.c_void_p), ("ndirty", ctypes.c_int64), ("first", ctypes.c_int64),
                ("count", ctypes.c_int64)]


PROPOSE = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.POINTER(View), ctypes.c_void_p,
                           ctypes.c_void_p, ctypes.c_void_p)


def _arr(addr, ctype, count):
    return np.ctypeslib.as_array((ctype * count).from_address(addr)).copy()


def test_view_layout_matches_header(tmp_path):
    fields = ["n", "d", "S", "M", "efc", "X", "level", "row0", "nrows", "adj", "adjd", "cnt", "entry_seg",
              "top_seg", "dirty", "ndirty", "first", "count"]
    prog = tmp_path / "v.c"
    prog.write_text('#include <stddef.h>\n#include <stdio.h>\n#include "unify.h"\nint main(void){'
                    'printf("%zu", sizeof(unify_build_view_t));'
                    + "".join(f'printf(" %zu", offsetof(unify_build_view_t, {f}));' for f in fields)
                    + "return 0;}\n")
    exe = tmp_path / "v"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    assert got == [ctypes.sizeof(View)] + [getattr(View, f).offset for f in fields]


def _first_assisted_batch(n):
    done = 0
    while done < n:
        bs = 1 if done < 1024 else min(4096, done // 64)
        if bs >= 64:
            return done, min(bs, n - done)
        done = min(n, done + bs)
    return None


def test_first_callback_sees_the_whole_graph_and_errors_propagate(tmp_path):
    rng = np.random.default_rng(3)
    n, d, S, M, efc = 4400, 8, 4, 8, 24
    x = rng.integers(0, 16, size=(n, d)).astype(np.float32)
    a = rng.permutation(n).astype(np.int64)
    seen = []

    def cb(ctx, view, out_ids, out_dist, out_cnt):
        v = view.contents
        nrows = v.nrows
        cnt = _arr(v.cnt, ctypes.c_uint8, nrows * v.S)
        dirty = _arr(v.dirty, ctypes.c_int64, v.ndirty) if v.ndirty else np.zeros(0, np.int64)
        level = _arr(v.level, ctypes.c_int32, v.n)
        row0 = _arr(v.row0, ctypes.c_int64, v.n)
        entry = _arr(v.entry_seg, ctypes.c_int32, v.S)
        top = _arr(v.top_seg, ctypes.c_int32, v.S)
        seen.append(dict(first=v.first, count=v.count, n=v.n, d=v.d, S=v.S, M=v.M, efc=v.efc, cnt=cnt,
                         dirty=dirty, level=level, row0=row0, entry=entry, top=top, nrows=nrows))
        return 7

    fn = PROPOSE(cb)
    with pytest.raises(RuntimeError, match=r"\(-3\).*code 7"):
        hsig_build.build_index(x, a, str(tmp_path / "g.idx"), S, M, efc, seed=5,
                               assist=(ctypes.cast(fn, ctypes.c_void_p).value, None, None, None))
    assert len(seen) == 1
    s = seen[0]
    first, count = _first_assisted_batch(n)
    assert (s["first"], s["count"]) == (first, count)
    assert (s["n"], s["d"], s["S"], s["M"], s["efc"]) == (n, d, S, M, efc)
    assert np.array_equal(s["row0"], np.concatenate([[0], np.cumsum(s["level"] + 1)[:-1]]))
    assert s["nrows"] == int(np.sum(s["level"] + 1))
    # every chunk written so far is listed once, and nothing else
    assert len(np.unique(s["dirty"])) == len(s["dirty"])
    assert np.array_equal(np.sort(s["dirty"]), np.flatnonzero(s["cnt"] > 0))
    # rows of nodes not yet inserted are empty
    assert not s["cnt"].reshape(-1, S)[s["row0"][first]:].any()
    # entry points: inserted nodes of their own segment, at the segment's top level
    for j in range(S):
        e = int(s["entry"][j])
        assert 0 <= e < first and s["top"][j] == s["level"][e]


def test_assisted_build_is_exact_bound():
    import paper_2412_02448_gb300 as U
    lo_hi = np.zeros((2, 258), np.float32)
    lo_hi[1] = 255.0
    assert U.assisted_build_is_exact(lo_hi)  # 258 * 255^2 < 2^24
    wide = np.zeros((2, 259), np.float32)
    wide[1] = 255.0
    assert not U.assisted_build_is_exact(wide)  # 259 * 255^2 >= 2^24
    half = lo_hi.copy()
    half[0, 7] = 0.5
    assert not U.assisted_build_is_exact(half)
    assert not U.assisted_build_is_exact(np.zeros((0, 4), np.float32))


APPLY = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.POINTER(View), ctypes.c_void_p, ctypes.c_void_p,
                         ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p)
FETCH = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.POINTER(View), ctypes.c_void_p, ctypes.c_void_p,
                         ctypes.c_void_p)


def test_device_owned_graph_protocol(tmp_path):
    """With apply and fetch, every batch from the first proposal on (the last, short one
    included) is proposed and applied by the callee, in strict alternation; apply gets
    the reverse edges of the proposals grouped by target chunk (ascending) in source-id
    order; fetch runs once, at the end, and its graph is what the file holds."""
    rng = np.random.default_rng(4)
    n, d, S, M, efc = 4300, 4, 2, 4, 8
    x = rng.integers(0, 8, size=(n, d)).astype(np.float32)
    a = rng.permutation(n).astype(np.int64)
    calls, snap = [], {}

    def propose(ctx, view, out_ids, out_dist, out_cnt):
        v = view.contents
        level = _arr(v.level, ctypes.c_int32, v.n)
        row0 = _arr(v.row0, ctypes.c_int64, v.n)
        if not snap:
            snap.update(adj=_arr(v.adj, ctypes.c_int32, v.nrows * S * M),
                        adjd=_arr(v.adjd, ctypes.c_float, v.nrows * S * M),
                        cnt=_arr(v.cnt, ctypes.c_uint8, v.nrows * S), nrows=v.nrows)
        rf = row0[v.first]
        last = v.first + v.count - 1
        rows = row0[last] + level[last] + 1 - rf
        cnt = np.zeros(rows * S, np.uint8)
        ids = np.zeros(rows * S * M, np.int32)
        dist = np.zeros(rows * S * M, np.float32)
        # one forward edge per node: layer 0, segment 0, to the node inserted just before the batch
        for t in range(v.count):
            e = (row0[v.first + t] - rf) * S
            cnt[e] = 1
            ids[e * M] = v.first - 1
            dist[e * M] = float(t + 1)
        ctypes.memmove(out_cnt, cnt.ctypes.data, cnt.nbytes)
        ctypes.memmove(out_ids, ids.ctypes.data, ids.nbytes)
        ctypes.memmove(out_dist, dist.ctypes.data, dist.nbytes)
        calls.append(("propose", v.first, v.count))
        return 0

    def apply(ctx, view, gc, gs, ng, rv, rd):
        v = view.contents
        g_chunk = _arr(gc, ctypes.c_int64, ng)
        g_start = _arr(gs, ctypes.c_int64, ng + 1)
        srcs = _arr(rv, ctypes.c_int32, g_start[-1])
        dists = _arr(rd, ctypes.c_float, g_start[-1])
        calls.append(("apply", v.first, v.count, g_chunk, g_start, srcs, dists))
        return 0

    def fetch(ctx, view, adj, adjd, cnt):
        calls.append(("fetch",))
        ctypes.memmove(adj, snap["adj"].ctypes.data, snap["adj"].nbytes)
        ctypes.memmove(adjd, snap["adjd"].ctypes.data, snap["adjd"].nbytes)
        ctypes.memmove(cnt, snap["cnt"].ctypes.data, snap["cnt"].nbytes)
        return 0

    fns = [PROPOSE(propose), APPLY(apply), FETCH(fetch)]
    path = hsig_build.build_index(x, a, str(tmp_path / "g.idx"), S, M, efc, seed=2,
                                  assist=tuple(ctypes.cast(f, ctypes.c_void_p).value for f in fns) + (None,))
    first, _ = _first_assisted_batch(n)
    assert calls[-1] == ("fetch",) and sum(c[0] == "fetch" for c in calls) == 1
    body = calls[:-1]
    assert [c[0] for c in body] == ["propose", "apply"] * (len(body) // 2)
    assert body[0][1] == first
    starts = [c[1] for c in body[0::2]]
    counts = [c[2] for c in body[0::2]]
    assert starts == list(np.cumsum([first] + counts[:-1])) and starts[-1] + counts[-1] == n
    assert counts[-1] < 64  # the short last batch stays with the callee
    for (_, f, c), (_, f2, c2, g_chunk, g_start, srcs, dists) in zip(body[0::2], body[1::2]):
        assert (f, c) == (f2, c2)
        assert g_start[0] == 0 and np.all(np.diff(g_start) > 0) and np.all(np.diff(g_chunk) > 0)
        # every batch node's single edge comes back, grouped by its segment's chunk of node f - 1
        assert sorted(srcs.tolist()) == list(range(f, f + c))
        for g in range(len(g_chunk)):
            s_ = srcs[g_start[g]:g_start[g + 1]]
            assert np.all(np.diff(s_) > 0)
            assert np.array_equal(dists[g_start[g]:g_start[g + 1]], (s_ - f + 1).astype(np.float32))
    # the file holds the fetched graph (the snapshot taken at the first proposal)
    g = hsig_build.read_index(path)
    adj = snap["adj"].reshape(snap["nrows"], S, M)
    row0 = np.concatenate([[0], np.cumsum(np.asarray(g["level"]) + 1)[:-1]])
    assert np.array_equal(np.asarray(g["adj0"]), adj[row0])


def test_build_index_dispatch(monkeypatch, tmp_path):
    """build_index takes the GPU-assisted builder whenever the assist's limits hold
    (integer or real-valued data), otherwise the host builder."""
    import paper_2412_02448_gb300 as U
    called = []
    monkeypatch.setattr(U, "build_index_gpu", lambda *a, **k: called.append("gpu") or a[2])
    monkeypatch.setattr(hsig_build, "build_index", lambda *a, **k: called.append("host") or a[2])
    ints = np.arange(40, dtype=np.float32).reshape(10, 4)
    attrs = np.arange(10, dtype=np.int64)
    cases = [(ints, 16, 100, "gpu"), (ints + 0.25, 16, 100, "gpu"), (ints, 40, 100, "host"),
             (ints, 16, 300, "host"), (np.zeros((10, 1100), np.float32), 16, 100, "host")]
    for x, M, efc, want in cases:
        called.clear()
        U.build_index(x, attrs, str(tmp_path / "i.idx"), 2, M, efc)
        assert called == [want], (M, efc, want)
