"""GPU-assisted construction (the proposal step of Algorithms 4 and 6 on the GPU).

On integer vectors whose squared distances stay below 2^24 both float32 distance
orders are exact, so the assisted build must write the same file, byte for byte, as
the host builder: this checks the device descent, ANNSearch, pruning and the
incremental upload of changed chunks together. On real-valued vectors the graphs may
differ by rounding; there the assisted index must be well-formed and search as well
as the host's."""
import os

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
    return U


def _same_file(a, b):
    with open(a, "rb") as f1, open(b, "rb") as f2:
        return f1.read() == f2.read()


def _case(name):
    from workloads import make_workload
    if name == "c2_int_d128":
        w = make_workload("c2", seed=7, n=30_000, nq=16)
        return w.vectors, w.attrs, w.S, w.M, w.efc
    rng = np.random.default_rng(11)
    n, d = 9_000, 200  # two float4 chunks per lane, ragged; duplicate attributes
    x = rng.integers(0, 24, size=(n, d)).astype(np.float32)
    a = rng.integers(0, 500, size=n).astype(np.int64)
    return x, a, 4, 8, 40


@pytest.mark.parametrize("name", ["c2_int_d128", "int_d200_dup_attrs"])
def test_assisted_build_equals_host_build(U, tmp_path, name):
    """Both modes: proposals only (the host applies edges and uploads changed chunks),
    and proposals plus edge application on the device (the graph fetched at the end)."""
    import hsig_build
    x, a, S, M, efc = _case(name)
    host = hsig_build.build_index(x, a, str(tmp_path / "host.idx"), S, M, efc, seed=3)
    for device_apply in (False, True):
        gpu = U.build_index_gpu(x, a, str(tmp_path / f"gpu{int(device_apply)}.idx"), S, M, efc, seed=3,
                                device_apply=device_apply)
        assert _same_file(host, gpu), device_apply


@pytest.mark.parametrize("shape", ["c1", "c4"])
def test_assisted_build_real_valued(U, tmp_path, shape):
    """On real-valued data (i.i.d. Gaussian; the unit-normalised mixture of the 10M
    precision shape) the assisted graph is well-formed (levels, segments and attribute
    order equal to the host build's; chunks hold distinct members of their segment) and
    its routed search recall is within 0.02 of the host-built graph's."""
    import hsig_build
    from workloads import make_workload
    w = make_workload(shape, seed=5, n=12_000, nq=200)
    host = hsig_build.build_index(w.vectors, w.attrs, str(tmp_path / "host.idx"), w.S, w.M, w.efc, seed=1)
    gpu = U.build_index_gpu(w.vectors, w.attrs, str(tmp_path / "gpu.idx"), w.S, w.M, w.efc, seed=1)
    g = hsig_build.read_index(gpu, verify=True)
    h = hsig_build.read_index(host, verify=True)
    for key in ("level", "seg_bounds", "sorted_ids"):
        assert np.array_equal(g[key], h[key]), key
    adj = np.asarray(g["adj0"])
    assert adj.min() >= -1 and adj.max() < w.n
    # chunk j holds only members of segment j, without duplicates
    seg = np.searchsorted(np.asarray(g["seg_bounds"])[1:-1], w.attrs, side="right")
    for v in range(0, w.n, 97):
        for j in range(w.S):
            ids = adj[v, j][adj[v, j] >= 0]
            assert np.all(seg[ids] == j) and len(set(ids.tolist())) == len(ids)
    ex = oracle.exact_knn(w.vectors, w.attrs, w.queries, w.lo, w.hi, w.k)
    p = U.Params.defaults(ef=64, ef_post=128, m=16)
    rec = {}
    for tag, path in (("host", host), ("gpu", gpu)):
        ix = U.Index(path)
        r = ix.search(w.queries, w.lo, w.hi, w.k, strategy="auto", params=p)
        torch.cuda.synchronize()
        rec[tag] = oracle.recall(r["ids"].cpu().numpy(), ex[0], ex[2], w.k).mean()
        ix.close()
    assert rec["gpu"] >= rec["host"] - 0.02


def test_assist_limits(U, tmp_path):
    rng = np.random.default_rng(2)
    n = 4_300  # the first batch of 64 nodes goes to the GPU after 4,096 host insertions
    x = rng.integers(0, 8, size=(n, 4)).astype(np.float32)
    a = np.arange(n, dtype=np.int64)
    with pytest.raises(U.UnifyError, match="M <= 32"):
        U.build_index_gpu(x, a, str(tmp_path / "m.idx"), 2, 40, 16)
    with pytest.raises(U.UnifyError, match="efc <= 256"):
        U.build_index_gpu(x, a, str(tmp_path / "e.idx"), 2, 8, 300)
    assert not os.path.exists(tmp_path / "m.idx")
