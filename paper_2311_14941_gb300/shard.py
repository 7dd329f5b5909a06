"""Cells over ranks: cost-balanced partition of a field and the one collective of the path.

Cells are independent reactors (Sec. 2.5), so integration shards with no data exchange: every rank
integrates its own cells.  Which cells a rank gets is decided from each cell's previous substep count,
the same cost key the sorted work queue uses, so that all ranks carry about the same work (the role of
the paper's load balancing between processes, Sec. 2.5): cells are taken in descending cost (ties by
index) and each goes to the rank with the least total so far (ties to the lowest rank): Graham's
longest-processing-time rule, whose spread between ranks never exceeds the largest single cost.
Every rank computes the same partition from the same cost array, so the partition itself needs no
communication.

The discrete adjoint's parameter gradients are sums over cells; ranks add theirs with one all-reduce of
2R doubles.  Timing takes the maximum over ranks.
"""
from __future__ import annotations

import numpy as np


def partition(cost, world: int) -> list:
    """Index arrays (ascending) of the cells of each of `world` ranks; together they cover every cell once."""
    if world < 1:
        raise ValueError("world must be >= 1")
    import heapq
    cost = np.asarray(cost, dtype=np.float64)
    n = cost.shape[0]
    order = np.lexsort((np.arange(n), -cost))
    owner = np.empty(n, dtype=np.int64)
    heap = [(0.0, r) for r in range(world)]
    for c in order.tolist():
        load, r = heapq.heappop(heap)
        owner[c] = r
        heapq.heappush(heap, (load + float(cost[c]), r))
    return [np.flatnonzero(owner == r) for r in range(world)]


def local_cells(cost, rank: int, world: int) -> np.ndarray:
    """This rank's share of `partition(cost, world)`."""
    if not 0 <= rank < world:
        raise ValueError("rank out of range")
    return partition(cost, world)[rank]


def allreduce_gradients(grad_lnA, grad_Ea, group=None) -> None:
    """Sums the per-rank parameter gradients over all ranks, in place (one collective of 2R values)."""
    import torch
    import torch.distributed as dist
    if not dist.is_initialized() or dist.get_world_size(group) == 1:
        return
    R = grad_lnA.numel()
    buf = torch.cat([grad_lnA.reshape(-1), grad_Ea.reshape(-1)])
    dist.all_reduce(buf, op=dist.ReduceOp.SUM, group=group)
    grad_lnA.copy_(buf[:R].view_as(grad_lnA))
    grad_Ea.copy_(buf[R:].view_as(grad_Ea))


def max_over_ranks(seconds: float, device=None, group=None) -> float:
    """The largest of the ranks' values (the job's time is its slowest rank's)."""
    import torch
    import torch.distributed as dist
    if not dist.is_initialized() or dist.get_world_size(group) == 1:
        return float(seconds)
    t = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())
