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
                ("cnt", ctypes.c_void_p), ("entry_seg", ctypes.c_void_p), ("top_seg", ctypes.c_void_p),
                ("dirty", ctypes.c_void_p), ("ndirty", ctypes.c_int64), ("first", ctypes.c_int64),
                ("count", ctypes.c_int64)]


PROPOSE = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.POINTER(View), ctypes.c_void_p,
                           ctypes.c_void_p, ctypes.c_void_p)


def _arr(addr, ctype, count):
    return np.ctypeslib.as_array((ctype * count).from_address(addr)).copy()


def test_view_layout_matches_header(tmp_path):
    fields = ["n", "d", "S", "M", "efc", "X", "level", "row0", "nrows", "adj", "cnt", "entry_seg",
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
                               propose=(ctypes.cast(fn, ctypes.c_void_p).value, None))
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
