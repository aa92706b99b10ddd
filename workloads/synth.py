"""Seeded synthetic workloads for range-filtered k-NN search.

This module only draws random numbers. It holds no distance, ranking, search or
graph arithmetic, so that both the CPU oracle and the CUDA path can be fed the
same inputs without sharing any of the method's code.

The shapes follow the datasets of the paper's evaluation (Section 5.1, Table 1):
SIFT1M (d=128, integer-valued descriptors), GIST1M (d=960, non-negative), GloVe
(d=100, unit-normalised). Those datasets are not available here, so these seeded
mixtures stand in for them. Attributes are integers; a query range is the
inclusive integer interval [lo, hi] (Definition 1, Section 2.1).

Range recipe: a range fraction f over an attribute domain of D values gives a
width w = max(1, round(f * D)); lo is uniform in [0, D - w] and hi = lo + w - 1.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Workload", "CONFIGS", "make_workload", "gaussian_iid", "int_mixture",
    "unit_mixture", "nonneg_mixture", "make_ranges", "log_uniform_fractions", "second_attribute",
    "query_batch",
]


@dataclass
class Workload:
    name: str
    vectors: np.ndarray          # (n, d) float32, row-major
    attrs: np.ndarray            # (n,) int64
    queries: np.ndarray          # (nq, d) float32
    lo: np.ndarray               # (nq,) int64, inclusive
    hi: np.ndarray               # (nq,) int64, inclusive
    fractions: np.ndarray        # (nq,) float64, the range fraction each query was drawn with
    k: int
    S: int
    M: int
    efc: int
    seed: int
    params: dict = field(default_factory=dict)
    centroids: np.ndarray | None = None  # mixture centroids the queries are drawn around

    @property
    def n(self) -> int:
        return int(self.vectors.shape[0])

    @property
    def d(self) -> int:
        return int(self.vectors.shape[1])


def gaussian_iid(rng: np.random.Generator, n: int, d: int) -> np.ndarray:
    return rng.standard_normal((n, d), dtype=np.float32)


def _mixture_points(rng, centroids, n, sigma, dtype=np.float32):
    nc, d = centroids.shape
    lab = rng.integers(0, nc, size=n)
    out = np.empty((n, d), dtype=np.float32)
    step = 1 << 16
    for s in range(0, n, step):
        e = min(n, s + step)
        out[s:e] = centroids[lab[s:e]] + sigma * rng.standard_normal((e - s, d), dtype=np.float32)
    return out


def int_mixture(rng, n, d, n_centroids=1000, sigma=20.0, centroids=None):
    """Integer-valued vectors in [0, 255] from a Gaussian mixture (SIFT-like).

    Every coordinate is an integer stored in float32, so squared L2 distances of
    d <= 128 coordinates stay below 2**24 and are exact in float32.
    """
    if centroids is None:
        centroids = rng.uniform(0.0, 255.0, size=(n_centroids, d)).astype(np.float32)
    x = _mixture_points(rng, centroids, n, sigma)
    np.rint(x, out=x)
    np.clip(x, 0.0, 255.0, out=x)
    return x, centroids


def unit_mixture(rng, n, d, n_centroids=500, sigma=0.35, centroids=None):
    """Unit-normalised Gaussian mixture (GloVe-like, inner-product workloads)."""
    if centroids is None:
        centroids = rng.standard_normal((n_centroids, d)).astype(np.float32)
        centroids /= np.linalg.norm(centroids, axis=1, keepdims=True)
    x = _mixture_points(rng, centroids, n, sigma / np.sqrt(d))
    x /= np.linalg.norm(x, axis=1, keepdims=True)
    return x.astype(np.float32), centroids


def nonneg_mixture(rng, n, d, n_centroids=1000, sigma=0.08, centroids=None):
    """Non-negative mixture with values in [0, 1] (GIST-like)."""
    if centroids is None:
        centroids = rng.uniform(0.0, 1.0, size=(n_centroids, d)).astype(np.float32) ** 2
    x = _mixture_points(rng, centroids, n, sigma)
    np.clip(x, 0.0, 1.0, out=x)
    return x, centroids


def make_ranges(rng, fractions: np.ndarray, domain: int):
    """Inclusive integer ranges of width max(1, round(f*domain)) at uniform offsets."""
    fractions = np.asarray(fractions, dtype=np.float64)
    w = np.maximum(1, np.rint(fractions * domain)).astype(np.int64)
    w = np.minimum(w, domain)
    lo = (rng.random(len(fractions)) * (domain - w + 1)).astype(np.int64)
    lo = np.minimum(lo, domain - w)
    hi = lo + w - 1
    return lo, hi


def log_uniform_fractions(rng, nq, lo_exp=-4.0, hi_exp=0.0):
    return 10.0 ** rng.uniform(lo_exp, hi_exp, size=nq)


# Workload configurations (sizes of the evaluated shapes). "frac" is a list of
# range fractions assigned round-robin to the queries, or "logu" for
# log-uniform fractions in [1e-4, 1].
CONFIGS = {
    "c1": dict(n=10_000, d=64, kind="gauss", attr="perm", S=8, M=16, efc=100,
               nq=200, frac=[0.01, 0.10, 0.50], k=10),
    "c2": dict(n=1_000_000, d=128, kind="int_mixture", centroids=1000, sigma=20.0,
               attr="uniform", domain=1_000_000, S=16, M=16, efc=100,
               nq=10_000, frac=[0.001, 0.01, 0.10, 0.50, 1.00], k=10),
    "c3": dict(n=1_000_000, d=96, kind="unit_mixture", centroids=500, attr="uniform",
               domain=1_000_000, S=8, M=16, efc=100, nq=10_000, frac="logu", k=10),
    "c4": dict(n=10_000_000, d=96, kind="unit_mixture", centroids=500, attr="uniform",
               domain=10_000_000, S=8, M=16, efc=100, nq=10_000,
               frac=[0.01, 0.10, 0.50], k=10),
    "c5": dict(n=1_000_000, d=960, kind="nonneg_mixture", centroids=1000,
               attr="uniform", domain=1_000_000, S=8, M=16, efc=100, nq=5_000,
               frac=[0.005, 0.02, 0.10], k=10),
}


def second_attribute(n: int, fractions, seed: int, domain: int = 1000):
    """A second integer attribute, uniform in [0, domain), and one range per query on
    it (width max(1, round(f * domain)) for each fraction f, start uniform), for
    conjunctive queries. Returns (attr2 int64 [n], lo2 int64 [nq], hi2 int64 [nq])."""
    rng = np.random.default_rng([seed, 5])
    attr2 = rng.integers(0, domain, size=n, dtype=np.int64)
    lo2, hi2 = make_ranges(rng, np.asarray(fractions, dtype=np.float64), domain)
    return attr2, lo2, hi2


def make_workload(name: str, seed: int = 1234, **overrides) -> Workload:
    """Build a seeded workload. Keyword overrides replace config fields
    (e.g. n=20_000, nq=64 for a small case of the same shape)."""
    if name not in CONFIGS:
        raise KeyError(f"unknown workload {name!r}; known: {sorted(CONFIGS)}")
    cfg = dict(CONFIGS[name])
    cfg.update(overrides)
    n, d, nq = int(cfg["n"]), int(cfg["d"]), int(cfg["nq"])
    rng_base = np.random.default_rng([seed, 0])
    rng_attr = np.random.default_rng([seed, 1])
    rng_q = np.random.default_rng([seed, 2])
    rng_r = np.random.default_rng([seed, 3])

    kind = cfg["kind"]
    c = None
    if kind == "gauss":
        x = gaussian_iid(rng_base, n, d)
    elif kind == "int_mixture":
        x, c = int_mixture(rng_base, n, d, cfg.get("centroids", 1000), cfg.get("sigma", 20.0))
    elif kind == "unit_mixture":
        x, c = unit_mixture(rng_base, n, d, cfg.get("centroids", 500))
    elif kind == "nonneg_mixture":
        x, c = nonneg_mixture(rng_base, n, d, cfg.get("centroids", 1000))
    else:
        raise ValueError(kind)

    if cfg["attr"] == "perm":
        attrs = rng_attr.permutation(n).astype(np.int64)
        domain = n
    else:
        domain = int(cfg.get("domain", n))
        attrs = rng_attr.integers(0, domain, size=n, dtype=np.int64)

    params = {k_: v for k_, v in cfg.items() if k_ not in ("n", "d", "nq")}
    params["domain"] = domain
    q, lo, hi, fr = _draw_queries(cfg, c, d, nq, domain, rng_q, rng_r)
    return Workload(name=name, vectors=np.ascontiguousarray(x, dtype=np.float32),
                    attrs=attrs, queries=q, lo=lo, hi=hi, fractions=fr, k=int(cfg["k"]), S=int(cfg["S"]),
                    M=int(cfg["M"]), efc=int(cfg["efc"]), seed=seed, params=params, centroids=c)


def _draw_queries(cfg, centroids, d, nq, domain, rng_q, rng_r):
    """Query vectors (around the base set's centroids, or N(0, 1) for the i.i.d.
    shape) and their ranges, by the workload's recipe."""
    kind = cfg["kind"]
    if kind == "gauss":
        q = gaussian_iid(rng_q, nq, d)
    elif kind == "int_mixture":
        q, _ = int_mixture(rng_q, nq, d, centroids=centroids, sigma=cfg.get("sigma", 20.0))
    elif kind == "unit_mixture":
        q, _ = unit_mixture(rng_q, nq, d, centroids=centroids)
    else:
        q, _ = nonneg_mixture(rng_q, nq, d, centroids=centroids)
    if cfg["frac"] == "logu":
        fr = log_uniform_fractions(rng_r, nq)
    else:
        fl = np.asarray(cfg["frac"], dtype=np.float64)
        fr = fl[np.arange(nq) % len(fl)]
    lo, hi = make_ranges(rng_r, fr, domain)
    return np.ascontiguousarray(q, dtype=np.float32), lo, hi, fr


def query_batch(w: Workload, query_seed: int, nq: int | None = None):
    """Another batch of queries for the base set of ``w``, drawn by the same recipe
    from an independent stream (``query_seed``): a held-out batch for tuning.
    Returns (queries, lo, hi, fractions)."""
    cfg = dict(CONFIGS[w.name])
    cfg.update({k_: v for k_, v in w.params.items() if k_ in cfg})
    nq = int(nq if nq is not None else len(w.lo))
    return _draw_queries(cfg, w.centroids, w.d, nq, int(w.params["domain"]),
                         np.random.default_rng([query_seed, 2]), np.random.default_rng([query_seed, 3]))
