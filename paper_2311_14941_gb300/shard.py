"""Cells over ranks: cost-balanced partition of a field and the one collective of the path.

Cells are independent reactors (Sec. 2.5), so integration shards with no data exchange: every rank
integrates its own cells.  Which cells a rank gets is decided from each cell's previous substep count,
the same cost key the sorted work queue uses, so that all ranks carry about the same work (the role of
the paper's load balancing between processes, Sec. 2.5): cells are taken in descending cost (ties by
index) and each goes to the rank with the least total so far (ties to the lowest rank): Graham's
longest-processing-time rule, whose spread between ranks never exceeds the largest single cost.
Every rank computes the same partition from the same cost array, so the partition itself needs no
communication.

When each rank owns its own cells (a CFD domain decomposition), the same balance needs data movement:
`Exchange` asks the library's planner (chem_balance_plan) where every cell should be integrated, sends
the states there with one all-to-all and returns the results with another; `balanced_integrate` wraps
one chemistry step in it.  This is the paper's dynamic load balancing between processes (Sec. 2.5).

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


def _comm_device(group=None):
    """The device a collective of `group` takes its tensors on: the current GPU for NCCL, else the CPU."""
    import torch
    import torch.distributed as dist
    if dist.get_backend(group) == "nccl":
        return torch.device("cuda", torch.cuda.current_device())
    return torch.device("cpu")


def gather_costs(cost_local, group=None) -> list:
    """Every rank's per-cell cost array, in rank order (an all-gather of the counts, then one of the
    costs padded to the longest)."""
    import torch
    import torch.distributed as dist
    cost_local = np.asarray(cost_local, dtype=np.float64)
    if not dist.is_initialized() or dist.get_world_size(group) == 1:
        return [cost_local]
    world = dist.get_world_size(group)
    dev = _comm_device(group)
    n = torch.tensor([cost_local.shape[0]], dtype=torch.int64, device=dev)
    ns = [torch.empty_like(n) for _ in range(world)]
    dist.all_gather(ns, n, group=group)
    counts = [int(x.item()) for x in ns]
    width = max(max(counts), 1)
    buf = torch.zeros(width, dtype=torch.float64, device=dev)
    buf[:cost_local.shape[0]] = torch.as_tensor(cost_local, device=dev)
    bufs = [torch.empty_like(buf) for _ in range(world)]
    dist.all_gather(bufs, buf, group=group)
    return [b[:c].cpu().numpy() for b, c in zip(bufs, counts)]


class Exchange:
    """Where this rank's cells are integrated and how their states travel.

    Built from the local cells' costs (previous substep counts; 1 where unknown).  All ranks gather all
    costs and run the same deterministic plan (chem_balance_plan), so they agree on it without further
    messages.  `forward` sends rows of cell data (one row per local cell) to the ranks that integrate
    them and returns this rank's work rows, ordered by source rank and then by the source's local index
    (this rank's own kept cells come in the same position as any other source's).  `backward` returns
    work rows to their owners and restores the local order.  One all-to-all each way; rows may differ in
    width between the two directions."""

    def __init__(self, cost_local, group=None):
        import torch.distributed as dist
        from . import chem
        self.group = group
        self.dist = dist.is_initialized() and dist.get_world_size(group) > 1
        self.rank = dist.get_rank(group) if self.dist else 0
        self.world = dist.get_world_size(group) if self.dist else 1
        costs = gather_costs(cost_local, group)
        self.counts = np.array([c.shape[0] for c in costs], dtype=np.int64)
        first = np.concatenate([[0], np.cumsum(self.counts)])
        dest_all = chem.balance_plan(self.counts, np.concatenate(costs) if len(costs) else np.zeros(0))
        self.dest_all = dest_all
        self.loads = np.bincount(dest_all, weights=np.concatenate(costs), minlength=self.world)
        dest = dest_all[first[self.rank]:first[self.rank + 1]]
        self.dest = dest
        self.send_order = np.argsort(dest, kind="stable")          # by destination, then local index
        self.send_counts = np.bincount(dest, minlength=self.world).astype(np.int64)
        self.recv_counts = np.array([int(np.count_nonzero(dest_all[first[s]:first[s + 1]] == self.rank))
                                     for s in range(self.world)], dtype=np.int64)
        self.n_local = int(self.counts[self.rank])
        self.n_work = int(self.recv_counts.sum())
        self.moved_out = int(np.count_nonzero(dest != self.rank))

    def _a2a(self, x, out_rows, in_split, out_split):
        import torch
        import torch.distributed as dist
        out = torch.empty((out_rows,) + tuple(x.shape[1:]), dtype=x.dtype, device=x.device)
        if x.shape[1] == 0:
            return out
        dist.all_to_all_single(out, x.contiguous(), [int(v) for v in out_split], [int(v) for v in in_split],
                               group=self.group)
        return out

    def forward(self, rows):
        """rows [n_local, W] (this rank's cells in local order) -> [n_work, W] (the cells to integrate here)."""
        import torch
        if rows.shape[0] != self.n_local:
            raise ValueError(f"forward expects {self.n_local} rows, got {rows.shape[0]}")
        if not self.dist:
            return rows.clone()
        order = torch.as_tensor(self.send_order, device=rows.device)
        return self._a2a(rows.index_select(0, order), self.n_work, self.send_counts, self.recv_counts)

    def backward(self, rows):
        """rows [n_work, W] (results, in forward's order) -> [n_local, W] in local order."""
        import torch
        if rows.shape[0] != self.n_work:
            raise ValueError(f"backward expects {self.n_work} rows, got {rows.shape[0]}")
        if not self.dist:
            return rows.clone()
        back = self._a2a(rows, self.n_local, self.recv_counts, self.send_counts)
        out = torch.empty_like(back)
        out.index_copy_(0, torch.as_tensor(self.send_order, device=rows.device), back)
        return out


def balanced_integrate(integrate, n_species, T, p, Y, dt, h_io, nsub, status, group=None):
    """One chemistry step of this rank's cells, with the load balanced over all ranks.

    `integrate(T, p, Y, dt, h_io, nsub, status)` integrates a batch in place with chem_integrate's
    arguments and layouts (for example ``functools.partial(mech.integrate, rtol=1e-6)``); it is called once
    on the cells this rank was given (not at all if none).  The local arrays (Y species-major, [n*N])
    receive their own cells' results as if they had been integrated here; nsub's incoming values are the
    costs of the plan.  Tensors live where the process group's collectives take them (the GPU for NCCL,
    the CPU for gloo).  Returns the Exchange used."""
    import torch
    N = T.numel()
    n = int(n_species)
    cost = np.maximum(nsub.detach().cpu().numpy().astype(np.float64), 1.0)
    ex = Exchange(cost, group)
    f64 = torch.float64
    rows = torch.cat([T.view(N, 1), p.view(N, 1), dt.view(N, 1), h_io.view(N, 1), nsub.to(f64).view(N, 1),
                      Y.view(n, N).t()], dim=1)
    work = ex.forward(rows)
    M = ex.n_work
    Tw, pw, dtw, hw = (work[:, j].contiguous() for j in range(4))
    nsw = work[:, 4].to(torch.int32).contiguous()
    Yw = work[:, 5:].t().contiguous().view(-1)
    stw = torch.zeros(M, dtype=torch.int32, device=T.device)
    if M > 0:
        integrate(Tw, pw, Yw, dtw, hw, nsw, stw)
    res = ex.backward(torch.cat([Tw.view(M, 1), hw.view(M, 1), nsw.to(f64).view(M, 1), stw.to(f64).view(M, 1),
                                 Yw.view(n, M).t()], dim=1))
    T.copy_(res[:, 0])
    h_io.copy_(res[:, 1])
    nsub.copy_(res[:, 2].to(torch.int32))
    status.copy_(res[:, 3].to(torch.int32))
    Y.view(n, N).copy_(res[:, 4:].t())
    return ex
