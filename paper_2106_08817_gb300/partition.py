"""Sharding one job of independent registrations across ranks (one GPU each).

Every registration problem (Eq. 4 cost and its gradient, Sec. 2-3 of
arXiv:2106.08817) is self-contained, so a job of many problems splits across
ranks with no exchange in the data path: each rank runs its share, and only
the scalar costs are gathered at the end, back in the job's instance order.

The split balances work measured in voxel-steps (voxels x T of a problem,
what one cost_and_grad moves through the forward and adjoint sweeps):
longest-processing-time-first list scheduling, each problem in turn (largest
first) to the rank with the least work so far.  Its makespan is at most
4/3 - 1/(3N) of the optimum (Graham's bound for LPT) and never more than the
mean load plus the largest problem.  Host code only; the collectives are
torch.distributed's (gloo on CPU, NCCL between GPUs).
"""
from __future__ import annotations

from typing import List, Sequence

__all__ = ["partition", "rank_share", "load_of", "gather_in_order"]


def partition(work: Sequence[float], nranks: int) -> List[List[int]]:
    """Instance indices per rank (each list ascending).  `work` is each instance's
    load (voxel-steps); ties go to the lower rank, so every rank computes the same
    split without communicating."""
    if nranks < 1:
        raise ValueError("nranks must be >= 1")
    if any(w < 0 for w in work):
        raise ValueError("work must be non-negative")
    order = sorted(range(len(work)), key=lambda i: (-work[i], i))
    load = [0.0] * nranks
    out: List[List[int]] = [[] for _ in range(nranks)]
    for i in order:
        r = min(range(nranks), key=lambda k: (load[k], k))
        out[r].append(i)
        load[r] += work[i]
    for lst in out:
        lst.sort()
    return out


def rank_share(work: Sequence[float], nranks: int, rank: int) -> List[int]:
    """This rank's instance indices."""
    return partition(work, nranks)[rank]


def load_of(work: Sequence[float], share: Sequence[int]) -> float:
    return float(sum(work[i] for i in share))


def gather_in_order(local_idx: Sequence[int], local_vals: Sequence, n_total: int,
                    group=None) -> list:
    """Every rank passes its instances' indices and values (e.g. the [3] cost terms of
    each); every rank gets the list of all n_total values in instance order.  Raises
    if an index is missing or given twice."""
    import torch.distributed as dist
    if len(local_idx) != len(local_vals):
        raise ValueError("one value per local index")
    world = dist.get_world_size(group)
    parts = [None] * world
    dist.all_gather_object(parts, (list(local_idx), list(local_vals)), group=group)
    out = [None] * n_total
    seen = [False] * n_total
    for idx, vals in parts:
        for i, v in zip(idx, vals):
            if not 0 <= i < n_total or seen[i]:
                raise ValueError("instance %d missing from the split or given twice" % i)
            seen[i] = True
            out[i] = v
    if not all(seen):
        raise ValueError("instances %s were not gathered" % [i for i, s in enumerate(seen) if not s])
    return out
