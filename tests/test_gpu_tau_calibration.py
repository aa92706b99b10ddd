"""Range-aware strategy selection calibrated as Section 4.2 describes: base objects
as queries with random ranges, run under Strategies A, B and C; the turning points
where pre- and post-filtering overtake hybrid filtering at a recall target give
tau_A and tau_B."""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def U():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2412_02448_gb300 as U
    assert torch.cuda.is_available()
    return U


def test_tau_calibration_turning_points(U, c1_index):
    """On the c1 shape: the per-bin table covers the sampled range sizes in ascending,
    disjoint bins; every beam recorded meets the recall target on its bin; the
    thresholds are the table's turning points, with pre-filtering chosen for the
    smallest ranges; and a held-out sample of base-object queries routed by them, with
    the recorded beams, meets the target within sampling noise, its pre-filter rows
    exactly."""
    from paper_2412_02448_gb300 import autotune
    w, path = c1_index
    ix = U.Index(path)
    dom = (int(w.attrs.min()), int(w.attrs.max()))
    target = 0.95
    ta, tb, table = autotune.calibrate_tau(ix, w.vectors, dom, w.k, target=target, n_sample=1024, bins=10,
                                           seed=1)
    print("calibrated tau", ta, tb, table)
    assert len(table) >= 6
    for a, b in zip(table[:-1], table[1:]):
        assert a["y_hi"] < b["y_lo"]
    # c1's attributes are a permutation of the domain: every range holds an object (Y >= 1)
    assert sum(r["queries"] for r in table) == 1024
    assert all(r["timed_rows"] >= 8192 for r in table)
    assert (ta, tb) == autotune.turning_points(table, ix.n)
    assert 0 < ta < tb <= ix.n + 1
    assert table[0]["ms_pre"] <= table[0]["ms_hybrid"]
    # held-out base-object queries (another seed), routed by the calibrated thresholds
    p = autotune.calibrated_params(U.Params.defaults(), ta, tb, table)
    rng = np.random.default_rng([2, 77])
    ids = rng.choice(ix.n, size=600, replace=False)
    span = dom[1] - dom[0] + 1
    width = np.maximum(1, np.rint(span * 10.0 ** rng.uniform(-np.log10(span), 0.0, size=len(ids)))).astype(np.int64)
    lo = dom[0] + (rng.random(len(ids)) * (span - width + 1)).astype(np.int64)
    hi = lo + width - 1
    Q = w.vectors[ids]
    r = ix.search(Q, lo, hi, w.k, strategy="auto", params=p)
    torch.cuda.synchronize()
    ex_ids, _, ex_c = oracle.exact_knn(w.vectors, w.attrs, Q, lo, hi, w.k)
    rec = oracle.recall(r["ids"].cpu().numpy(), ex_ids, ex_c, w.k)
    Y = np.array([((w.attrs >= a) & (w.attrs <= b)).sum() for a, b in zip(lo, hi)])
    assert np.all(rec[Y <= ta] == 1.0)
    assert rec.mean() >= target - 0.02, rec.mean()
