"""Running independent region instances on several GPUs, one process each:
batches split by instance, served requests routed by load.

Teams share nothing across teams (each has its own stack, Sec. 4: a team
is a thread block), and region instances share nothing across instances.
So N GPUs split a set of instances by instance and need no collective on
the data path: each rank runs its share with its own launches, stacks and
overflow pool, and only the timing (the slowest rank) and, where wanted, a
host-side gather of outputs cross ranks. This module holds that host logic;
it works on any torch.distributed backend (gloo on CPU, nccl on GPUs).
"""
from __future__ import annotations

from typing import Dict, List, Sequence, Tuple

import numpy as np


def balanced_ranges(weights: Sequence[int], world: int) -> List[Tuple[int, int]]:
    """Split instances 0..n-1 into `world` contiguous ranges whose weights
    (team counts, say) are as even as prefix sums allow: rank r takes the
    instances whose weight prefix falls in [r*total/world, (r+1)*total/world).
    Every instance goes to exactly one rank; a rank may get none."""
    if world < 1:
        raise ValueError("world must be >= 1")
    w = np.asarray(weights, dtype=np.int64)
    if (w < 0).any():
        raise ValueError("weights must be non-negative")
    n = len(w)
    if n == 0:
        return [(0, 0)] * world
    # instance i belongs to the rank its weight's midpoint lands in
    before = np.concatenate([[0], np.cumsum(w)[:-1]])
    total = int(w.sum())
    if total == 0:
        owner = (np.arange(n) * world) // n
    else:
        mid2 = 2 * before + w  # twice the midpoint, kept integral
        owner = np.minimum((mid2 * world) // (2 * total), world - 1)
    owner = np.maximum.accumulate(owner)  # contiguous and non-decreasing
    ranges = []
    for r in range(world):
        idx = np.nonzero(owner == r)[0]
        if len(idx):
            ranges.append((int(idx[0]), int(idx[-1]) + 1))
        else:
            start = ranges[-1][1] if ranges else 0
            ranges.append((start, start))
    return ranges


def route_requests(weights: Sequence[int], world: int) -> np.ndarray:
    """Serving on several GPUs: the rank (GPU) of each request, in arrival
    order, each to the rank with the least weight (teams, say) routed so far,
    ties to the lowest rank. The routing depends on the requests alone, so
    every rank computes the same one and keeps its own requests, with no
    message between ranks; every rank then serves its requests with its own
    server."""
    if world < 1:
        raise ValueError("world must be >= 1")
    w = np.asarray(weights, dtype=np.int64)
    if (w < 0).any():
        raise ValueError("weights must be non-negative")
    load = np.zeros(world, dtype=np.int64)
    rank = np.empty(len(w), dtype=np.int64)
    for i, x in enumerate(w.tolist()):
        r = int(np.argmin(load))
        rank[i] = r
        load[r] += x
    return rank


def _scalar_tensor(value: float, dist):
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    if dev == "cuda":
        dev = torch.device("cuda", torch.cuda.current_device())
    return torch.tensor([float(value)], dtype=torch.float64, device=dev)


def max_over_ranks(value: float, dist=None) -> float:
    """The largest `value` of all ranks (the step time of the slowest rank
    is the job's step time). Without an initialised process group: value."""
    if dist is None or not dist.is_initialized():
        return float(value)
    t = _scalar_tensor(value, dist)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float, dist=None) -> float:
    """The sum of `value` over ranks (units processed by the whole job)."""
    if dist is None or not dist.is_initialized():
        return float(value)
    t = _scalar_tensor(value, dist)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def gather_to_rank0(local: Dict[int, np.ndarray], dist=None):
    """Host gather of per-instance results keyed by global instance index:
    rank 0 receives the union of every rank's dict, the others None. Keys
    must be disjoint across ranks."""
    if dist is None or not dist.is_initialized():
        return dict(local)
    world = dist.get_world_size()
    parts = [None] * world if dist.get_rank() == 0 else None
    dist.gather_object(local, parts, dst=0)
    if dist.get_rank() != 0:
        return None
    merged: Dict[int, np.ndarray] = {}
    for p in parts:
        for k, v in p.items():
            if k in merged:
                raise ValueError("instance %d reported by two ranks" % k)
            merged[k] = v
    return merged
