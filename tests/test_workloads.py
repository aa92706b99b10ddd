import numpy as np

from workloads import make_workload


def test_shapes_and_determinism():
    a = make_workload("c2", n=5000, nq=50, seed=3)
    b = make_workload("c2", n=5000, nq=50, seed=3)
    assert a.vectors.shape == (5000, 128) and a.queries.shape == (50, 128)
    assert np.array_equal(a.vectors, b.vectors) and np.array_equal(a.lo, b.lo)
    assert np.all(a.vectors == np.rint(a.vectors)) and a.vectors.min() >= 0 and a.vectors.max() <= 255


def test_range_widths():
    w = make_workload("c1", nq=300)
    width = w.hi - w.lo + 1
    assert np.array_equal(width, np.maximum(1, np.rint(w.fractions * w.n)).astype(np.int64))
    assert w.lo.min() >= 0 and w.hi.max() <= w.n - 1
    w3 = make_workload("c3", n=2000, nq=500)
    assert w3.fractions.min() >= 1e-4 and w3.fractions.max() <= 1.0
    assert np.allclose(np.linalg.norm(w3.vectors, axis=1), 1.0, atol=1e-5)
