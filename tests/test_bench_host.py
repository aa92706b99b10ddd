"""Host logic of bench.py (no GPU): the DRAM-traffic table lookup, the stratified
row sample, the clock-sample parsing and the truth check against the oracle's exact
range-filtered k-NN (Definition 1)."""
import os
import types

import numpy as np
import pytest

import bench

pytestmark = pytest.mark.filterwarnings("ignore")


def _params(**kw):
    p = types.SimpleNamespace()
    base = {k: 1 for k in bench.TRAFFIC_KEYS}
    base.update(kw)
    for k, v in base.items():
        setattr(p, k, v)
    return p


def test_traffic_table_entries_are_complete():
    """Every capture names a digest, a workload, positive bytes and every key the
    lookup compares."""
    for c in bench.NCU_TRAFFIC:
        assert len(c["digest"]) == 12 and c["workload"] in bench.WORKLOADS and c["bytes"] > 0
        assert set(bench.TRAFFIC_KEYS) <= set(c["params"]), c
        assert os.path.exists(os.path.join(bench.ROOT, c["profile"]))


def test_traffic_lookup_matches_digest_workload_and_every_parameter(monkeypatch):
    cap = {"digest": "abcdef012345", "workload": "c2", "bytes": 123,
           "params": {k: 7 for k in bench.TRAFFIC_KEYS}, "profile": "profiles/batch_kernel_c2_1m_launches.md"}
    monkeypatch.setattr(bench, "NCU_TRAFFIC", [cap])
    assert bench.traffic_for("abcdef012345", "c2", _params(**{k: 7 for k in bench.TRAFFIC_KEYS})) == (123, cap)
    # one parameter differs: no traffic, the nearest capture of the kernel and workload
    for k in bench.TRAFFIC_KEYS:
        p = _params(**{kk: 7 for kk in bench.TRAFFIC_KEYS})
        setattr(p, k, 8)
        assert bench.traffic_for("abcdef012345", "c2", p) == (None, cap), k
    # another kernel source or workload: nothing at all
    assert bench.traffic_for("000000000000", "c2", _params(**{k: 7 for k in bench.TRAFFIC_KEYS})) == (None, None)
    assert bench.traffic_for("abcdef012345", "c4", _params(**{k: 7 for k in bench.TRAFFIC_KEYS})) == (None, None)


def test_stratified_rows():
    fr = np.array([0.1, 0.5, 0.1, 0.5, 0.1, 1.0])
    assert bench.stratified_rows(fr, 0).tolist() == list(range(6))
    assert bench.stratified_rows(fr, 1).tolist() == [0, 1, 5]
    assert bench.stratified_rows(fr, 2).tolist() == [0, 1, 2, 3, 5]


def test_clock_samples_parse(tmp_path, monkeypatch):
    """The nvidia-smi CSV the bench samples: median SM clock, maximum, the throttle
    reasons seen active."""
    monkeypatch.setenv("UNIFY_CACHE_DIR", str(tmp_path))
    c = bench.Clocks(0)
    rows = ["0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
            "0, 2000, 2070, 1300.0, 0x4, Not Active, Not Active, Not Active, Active",
            "0, 2070, 2070, 950.0, 0x0, Not Active, Not Active, Not Active, Not Active"]
    with open(c.path, "w") as f:
        f.write("\n".join(rows) + "\n")

    class Done:
        def terminate(self):
            pass

        def wait(self, timeout=None):
            return 0

    c.proc = Done()
    c.f = open(os.devnull, "w")
    r = c.stop()
    assert r["sm_mhz"] == 2070.0 and r["sm_max_mhz"] == 2070.0 and r["samples"] == 3
    assert r["reasons"] == ["sw_power_cap"]


def test_truth_check_counts_equal_tie_band_and_mismatch():
    """Rows equal to the oracle's exact answer count as equal; a swap of two objects at
    the same FP64 distance as the k-th counts as a tie-band swap; a wrong id as a
    mismatch."""
    import oracle
    rng = np.random.default_rng(3)
    n, d, k = 400, 8, 5
    X = rng.standard_normal((n, d)).astype(np.float32)
    # object 1 duplicates object 0: the two are at the same distance from any query
    X[1] = X[0]
    attrs = np.arange(n, dtype=np.int64)
    Q = rng.standard_normal((3, d)).astype(np.float32)
    lo = np.zeros(3, np.int64)
    hi = np.full(3, n - 1, np.int64)
    # query 1 sits on object 0, so objects 0 and 1 are its two nearest (distance 0)
    Q[1] = X[0]
    ex_ids, ex_d, ex_c = oracle.exact_knn(X, attrs, Q, lo, hi, k)
    w = types.SimpleNamespace(vectors=X, attrs=attrs, queries=Q, lo=lo, hi=hi,
                              fractions=np.array([1.0, 1.0, 1.0]))
    rows = np.arange(3)
    t_ids = ex_ids.copy()
    t_cnt = ex_c.copy()
    r = bench.truth_check(w, rows, t_ids, t_cnt, k, per_fraction=3)
    assert r == {"rows": 3, "ids_equal": 3, "tie_band_swaps": 0, "mismatch": 0}
    # query 1: objects 0 and 1 tie at distance 0 and rank first and second; with k = 1
    # the exact answer holds one of them, and the other is an equally valid answer
    ex1, _, c1 = oracle.exact_knn(X, attrs, Q, lo, hi, 1)
    t1 = ex1.copy()
    t1[1, 0] = 1 - ex1[1, 0]
    r = bench.truth_check(w, rows, t1, c1, 1, per_fraction=3)
    assert r["ids_equal"] == 2 and r["tie_band_swaps"] == 1 and r["mismatch"] == 0
    # a far object in place of the k-th: a mismatch
    t2 = ex_ids.copy()
    far = np.argmax(((X.astype(np.float64) - Q[2].astype(np.float64)) ** 2).sum(1))
    t2[2, k - 1] = far
    r = bench.truth_check(w, rows, t2, t_cnt, k, per_fraction=3)
    assert r["mismatch"] == 1 and r["ids_equal"] == 2
    # a count that differs: a mismatch
    t3 = t_cnt.copy()
    t3[0] -= 1
    r = bench.truth_check(w, rows, t_ids, t3, k, per_fraction=3)
    assert r["mismatch"] == 1
