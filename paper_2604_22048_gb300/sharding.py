"""Host logic for running the path on several GPUs (one process per GPU).

The image sampling phase shards by galaxy with no exchange; the shear
likelihood (Eq. likelihood-shear) is a sum over galaxies, so each rank
evaluates its share and the 4 doubles (value, d/dg1, d/dg2, d/dalpha) are
summed across ranks once per evaluation.
"""
from __future__ import annotations

import heapq

import numpy as np


def galaxy_cost(side):
    """Relative cost of fitting one galaxy: one pass over the (N+1)/2 x N
    half-plane spectrum per gradient evaluation."""
    side = np.asarray(side, dtype=np.int64)
    return (side + 1) // 2 * side


def partition_galaxies(side, world):
    """Greedy size-balanced assignment (largest first to the least-loaded
    rank).  Returns a list of index arrays, one per rank, each sorted."""
    cost = galaxy_cost(side)
    order = np.argsort(-cost, kind="stable")
    heap = [(0, r) for r in range(world)]
    parts = [[] for _ in range(world)]
    for i in order:
        load, r = heapq.heappop(heap)
        parts[r].append(int(i))
        heapq.heappush(heap, (load + int(cost[i]), r))
    return [np.array(sorted(p), dtype=np.int64) for p in parts]


def make_allreduce(group=None, device=None):
    """Callable summing a length-4 float64 numpy vector over the process
    group (torch.distributed: gloo on CPU tensors, NCCL on CUDA tensors)."""
    import torch
    import torch.distributed as dist

    buf = torch.zeros(4, dtype=torch.float64, device=device)

    def allreduce(x):
        buf.copy_(torch.as_tensor(np.asarray(x, dtype=np.float64)))
        dist.all_reduce(buf, group=group)
        return buf.cpu().numpy()

    return allreduce
