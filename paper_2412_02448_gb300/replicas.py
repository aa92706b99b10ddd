"""Multi-GPU execution of a search batch: replicas only.

Queries are independent and the index fits one GPU, so N GPUs run N replicas of
the index, each searching its own batch of the same shape (weak scaling). The
only collectives are a barrier around the timed region and the max-reduction of
the per-rank step time; there is no collective on the data path.
"""
from __future__ import annotations

import numpy as np


def rank_batch(queries, lo, hi, fractions, rank: int, seed: int):
    """The batch searched by `rank`: rank 0 keeps the given order, other ranks a
    seeded permutation of it (same size and range-fraction mix)."""
    if rank == 0:
        return queries, lo, hi, fractions
    perm = np.random.default_rng([seed, 100 + rank]).permutation(len(lo))
    return queries[perm], lo[perm], hi[perm], fractions[perm]


def max_over_ranks(value: float, world: int, device=None) -> float:
    """Maximum of a per-rank scalar (the step time) over all ranks."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_qps(queries_per_rank: int, world: int, ms_max: float) -> float:
    """Whole-job throughput: every rank's queries over the slowest rank's time."""
    return world * queries_per_rank / (ms_max / 1000.0)
