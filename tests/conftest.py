import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
TESTS = os.path.dirname(os.path.abspath(__file__))
if TESTS not in sys.path:
    sys.path.insert(0, TESTS)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the compiled CUDA library")


def cache_dir():
    d = os.environ.get("UNIFY_CACHE_DIR", os.path.join(ROOT, "_cache"))
    os.makedirs(d, exist_ok=True)
    return d


def built_index(name, seed=7, **overrides):
    """Build (or reuse) the index of a seeded workload; returns (workload, path)."""
    from workloads import make_workload
    import hsig_build
    w = make_workload(name, seed=seed, **overrides)
    tag = "_".join(f"{k}{v}" for k, v in sorted(overrides.items()))
    path = os.path.join(cache_dir(), f"{name}_s{seed}_{tag}_{hsig_build.source_digest()}.idx")
    if not os.path.exists(path):
        hsig_build.build_index(w.vectors, w.attrs, path, w.S, w.M, w.efc, seed=seed)
    return w, path


@pytest.fixture(scope="session")
def c1_index():
    return built_index("c1")


@pytest.fixture(scope="session")
def c2_small_index():
    """c2-shaped (integer-valued, d=128, S=16) at n = 20,000: float32 distances are exact."""
    return built_index("c2", n=20_000, nq=300)


@pytest.fixture(scope="session")
def c3_small_index():
    """GloVe-like shape: d = 96 unit vectors, log-uniform range fractions."""
    return built_index("c3", n=20_000, nq=200)


@pytest.fixture(scope="session")
def c4_small_index():
    """The 10M precision shape (unit-normalised d = 96 mixture, ranges 1/10/50 %) at
    n = 20,000."""
    return built_index("c4", n=20_000, nq=150)


@pytest.fixture(scope="session")
def c5_small_index():
    """GIST-like shape: d = 960 non-negative values in [0, 1]."""
    return built_index("c5", n=6_000, nq=120, efc=60)
