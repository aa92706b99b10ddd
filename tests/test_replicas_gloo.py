"""The multi-GPU path of the benchmark (replicas, weak scaling) on two gloo ranks on
the CPU: per-rank batches, the max-over-ranks step time and the whole-job rate."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2412_02448_gb300 import replicas
    from workloads import make_workload
    w = make_workload("c1", nq=60)
    q, lo, hi, fr = replicas.rank_batch(w.queries, w.lo, w.hi, w.fractions, rank, seed=5)
    local_ms = 10.0 + 5.0 * rank
    ms_max = replicas.max_over_ranks(local_ms, world)
    qps = replicas.aggregate_qps(len(lo), world, ms_max)
    out[rank] = (ms_max, qps, lo.tolist(), sorted(np.round(fr, 6).tolist()))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_replicas():
    world = 2
    mgr = mp.get_context("spawn").Manager()  # no fork of a possibly CUDA-initialised parent
    out = mgr.dict()
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    (m0, q0, lo0, f0), (m1, q1, lo1, f1) = out[0], out[1]
    assert m0 == m1 == 15.0                     # the slowest rank's time on every rank
    assert q0 == q1 == pytest.approx(2 * 60 / 0.015)
    assert sorted(lo0) == sorted(lo1) and lo0 != lo1  # same batch, each rank its own order
    assert f0 == f1                             # same range-fraction mix
