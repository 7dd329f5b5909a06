"""Load balancing between processes (the paper's DLB, Sec. 2.5): the library's planner
(chem_balance_plan) against a plain restatement of its rule and the bounds the rule guarantees, and
gloo runs on CPU of the exchange that moves cell states to the planned ranks and the results back."""
import heapq
import os
import socket

import numpy as np
import pytest

from paper_2311_14941_gb300 import chem, shard


def rule(costs_per_rank):
    """The planning rule written out directly: keep the cheapest prefix within the mean, then deal the
    rest in descending cost to the least-loaded rank."""
    world = len(costs_per_rank)
    total = sum(float(np.sum(c)) for c in costs_per_rank)
    target = total / world
    dest = [np.full(len(c), -1) for c in costs_per_rank]
    load = [0.0] * world
    pool = []
    for r, c in enumerate(costs_per_rank):
        order = sorted(range(len(c)), key=lambda i: (c[i], i))
        s = 0.0
        k = 0
        while k < len(order) and s + c[order[k]] <= target:
            s += c[order[k]]
            dest[r][order[k]] = r
            k += 1
        load[r] = s
        pool += [(c[i], r, i) for i in order[k:]]
    pool.sort(key=lambda t: (-t[0], t[1], t[2]))
    heap = [(load[r], r) for r in range(world)]
    heapq.heapify(heap)
    for cost, r, i in pool:
        l, q = heapq.heappop(heap)
        dest[r][i] = q
        heapq.heappush(heap, (l + cost, q))
    return dest


def plan(costs_per_rank):
    counts = [len(c) for c in costs_per_rank]
    flat = np.concatenate([np.asarray(c, dtype=np.float64) for c in costs_per_rank]) if counts else np.zeros(0)
    d = chem.balance_plan(counts, flat)
    first = np.concatenate([[0], np.cumsum(counts)])
    return [d[first[r]:first[r + 1]] for r in range(len(counts))]


def loads(costs_per_rank, dest, world):
    out = np.zeros(world)
    for c, d in zip(costs_per_rank, dest):
        np.add.at(out, d, c)
    return out


@pytest.mark.parametrize("world,seed", [(1, 0), (2, 1), (3, 2), (4, 3), (8, 4), (5, 5)])
def test_plan_is_the_rule_and_meets_its_bounds(world, seed):
    rng = np.random.default_rng(seed)
    # uneven ranks: different cell counts and a heavy-tailed cost, one rank much hotter than the rest
    costs = []
    for r in range(world):
        n = int(rng.integers(0, 400))
        c = np.maximum(1, rng.lognormal(2.0 + (1.5 if r == world // 2 else 0.0), 1.2, n)).round()
        costs.append(c)
    got = plan(costs)
    want = rule(costs)
    for g, w in zip(got, want):
        assert np.array_equal(g, w)
    total = sum(c.sum() for c in costs)
    target = total / world
    L = loads(costs, got, world)
    cmax = max((c.max() for c in costs if len(c)), default=0.0)
    assert abs(L.sum() - total) < 1e-9 * max(total, 1)
    assert L.max() <= target + cmax + 1e-9
    for r, (c, d) in enumerate(zip(costs, got)):
        assert np.all((d >= 0) & (d < world))
        if c.sum() <= target:
            assert np.all(d == r)          # an underloaded rank keeps everything
        else:
            kept = np.sort(c[d == r])
            # the kept cells are the longest cheapest prefix within the target: no more cells can stay
            srt = np.sort(c)
            k = np.searchsorted(np.cumsum(srt), target, side="right")
            assert len(kept) >= k


def test_plan_balances_a_skewed_field_within_one_cell():
    rng = np.random.default_rng(11)
    # rank 0 holds the flame (expensive cells), the others cold gas
    costs = [rng.integers(200, 2000, 5000).astype(float)] + [rng.integers(1, 4, 5000).astype(float)
                                                             for _ in range(3)]
    d = plan(costs)
    L = loads(costs, d, 4)
    assert L.max() - L.mean() <= max(c.max() for c in costs)
    assert L.max() / L.mean() < 1.001
    # the cold ranks send nothing
    for r in (1, 2, 3):
        assert np.all(d[r] == r)


def test_plan_edge_cases():
    assert plan([np.zeros(0), np.zeros(0)])[0].shape == (0,)
    z = plan([np.zeros(5), np.zeros(3)])                      # no cost anywhere: nothing moves
    assert np.all(z[0] == 0) and np.all(z[1] == 1)
    one = plan([np.array([7.0, 1.0, 1.0]), np.zeros(0)])      # all cells on one rank, the other empty
    L = loads([np.array([7.0, 1.0, 1.0]), np.zeros(0)], one, 2)
    assert sorted(L.tolist()) == [2.0, 7.0]


@pytest.mark.parametrize("args", [
    (0, [], []),
    (2, [3, -1], [1.0, 1.0]),
    (2, [1, 1], [1.0, float("nan")]),
    (2, [1, 1], [1.0, -2.0]),
    (1, [1], [float("inf")]),
])
def test_plan_rejects_bad_input(args):
    world, counts, costs = args
    import ctypes as C
    L = chem.lib()
    cnt = np.asarray(counts + [0] * (world - len(counts)), dtype=np.int64) if world else np.zeros(1, np.int64)
    cst = np.asarray(costs, dtype=np.float64)
    dest = np.zeros(max(len(costs), 1), dtype=np.int32)
    rc = L.chem_balance_plan(world, cnt.ctypes.data_as(C.c_void_p), cst.ctypes.data_as(C.c_void_p),
                             dest.ctypes.data_as(C.c_void_p))
    assert rc == 1
    assert L.chem_last_error()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _local_field(rank):
    """Rank r's own cells: different counts per rank (rank 1 has none), global ids and skewed costs."""
    sizes = [13, 0, 29]
    first = int(np.sum(sizes[:rank]))
    ids = np.arange(first, first + sizes[rank])
    cost = np.where(ids % 7 == 0, 500.0, 1.0 + ids % 3) * (3.0 if rank == 0 else 1.0)
    return ids, cost


def _exchange_main(rank, world, port, outdir):
    import torch
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        ids, cost = _local_field(rank)
        ex = shard.Exchange(cost)
        rows = torch.stack([torch.as_tensor(ids, dtype=torch.float64), torch.as_tensor(cost),
                            torch.full((len(ids),), float(rank), dtype=torch.float64)], 1) \
            if len(ids) else torch.zeros((0, 3), dtype=torch.float64)
        work = ex.forward(rows)
        # "integrate": results of a different width, tagged with the worker's rank
        res = torch.stack([work[:, 0] * 2.0 + 1.0, torch.full((work.shape[0],), float(rank), dtype=torch.float64)],
                          1) if work.shape[0] else torch.zeros((0, 2), dtype=torch.float64)
        back = ex.backward(res)
        np.savez(os.path.join(outdir, f"x{rank}.npz"), ids=ids, work_ids=work[:, 0].numpy(),
                 work_cost=work[:, 1].numpy(), work_src=work[:, 2].numpy(), back=back.numpy(), dest=ex.dest,
                 dest_all=ex.dest_all, loads=ex.loads, n_work=ex.n_work)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_three_gloo_ranks_exchange_cells_and_return_results(tmp_path):
    import torch.multiprocessing as mp
    world = 3
    mp.start_processes(_exchange_main, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       start_method="spawn", join=True)
    out = [np.load(tmp_path / f"x{r}.npz") for r in range(world)]
    for o in out[1:]:
        assert np.array_equal(o["dest_all"], out[0]["dest_all"])        # one plan on every rank
    costs = [_local_field(r)[1] for r in range(world)]
    want = plan(costs)
    assert np.array_equal(np.concatenate(want), out[0]["dest_all"])
    worked = np.concatenate([o["work_ids"] for o in out])
    assert np.array_equal(np.sort(worked), np.arange(42))                  # every cell integrated once
    for r, o in enumerate(out):
        # each worker received exactly the cells planned for it, in (source rank, local index) order
        planned = np.concatenate([_local_field(s)[0][want[s] == r] for s in range(world)])
        assert np.array_equal(o["work_ids"], planned)
        assert o["work_cost"].sum() == pytest.approx(o["loads"][r])
        # results came home in local order, computed by the planned rank
        ids = _local_field(r)[0]
        if len(ids):
            assert np.array_equal(o["back"][:, 0], ids * 2.0 + 1.0)
            assert np.array_equal(o["back"][:, 1], want[r].astype(np.float64))
    L = out[0]["loads"]
    allc = np.concatenate(costs)
    assert L.max() <= allc.sum() / world + allc.max()


def _integrate_main(rank, world, port, outdir):
    import functools
    import torch
    import torch.distributed as dist
    from oracle.oracle import Oracle
    from paper_2311_14941_gb300 import synth
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        m = synth.mechanism_small()
        F = synth.field_uniform_random(m, 30, seed=8)
        mine = np.arange(30)[:22] if rank == 0 else np.arange(30)[22:]     # rank 0 owns most of the field
        S = F.subset(mine)
        orc = Oracle(m)
        calls = []

        def integrate(T, p, Y, dt, h_io, nsub, status, rtol=1e-6, atol=1e-12):
            n, N = m.n_species, T.numel()
            r = orc.integrate_batch(T.numpy(), p.numpy(), Y.view(n, N).numpy(), dt.numpy(), rtol, atol,
                                    h_io=h_io.numpy(), nthreads=1)
            T.copy_(torch.as_tensor(r["T"]))
            Y.view(n, N).copy_(torch.as_tensor(r["Y"]))
            h_io.copy_(torch.as_tensor(r["h"]))
            nsub.copy_(torch.as_tensor(r["nsub"]))
            status.copy_(torch.as_tensor(r["status"]))
            calls.append(N)

        N = len(mine)
        T = torch.as_tensor(S.T.copy())
        p = torch.as_tensor(S.p.copy())
        Y = torch.as_tensor(S.Y.copy()).reshape(-1)
        dt = torch.as_tensor(S.dt.copy())
        h = torch.zeros(N, dtype=torch.float64)
        ns = torch.as_tensor(np.where(mine % 5 == 0, 40, 3).astype(np.int32))   # previous substep counts
        st = torch.zeros(N, dtype=torch.int32)
        ex = shard.balanced_integrate(functools.partial(integrate), m.n_species, T, p, Y, dt, h, ns, st)
        np.savez(os.path.join(outdir, f"i{rank}.npz"), cells=mine, T=T.numpy(), Y=Y.view(m.n_species, N).numpy(),
                 h=h.numpy(), nsub=ns.numpy(), status=st.numpy(), n_work=ex.n_work, moved=ex.moved_out,
                 calls=np.array(calls))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_balanced_integration_equals_local_integration(tmp_path):
    import torch.multiprocessing as mp
    from oracle.oracle import Oracle
    from paper_2311_14941_gb300 import synth
    world = 2
    mp.start_processes(_integrate_main, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       start_method="spawn", join=True)
    out = [np.load(tmp_path / f"i{r}.npz") for r in range(world)]
    assert int(out[0]["moved"]) > 0                     # the heavy rank really sent cells away
    assert int(out[0]["n_work"]) + int(out[1]["n_work"]) == 30
    m = synth.mechanism_small()
    F = synth.field_uniform_random(m, 30, seed=8)
    whole = Oracle(m).integrate_batch(F.T, F.p, F.Y, F.dt, 1e-6, 1e-12, nthreads=1)
    for o in out:
        c = o["cells"]
        assert np.array_equal(o["T"], whole["T"][c])
        assert np.array_equal(o["Y"], whole["Y"][:, c])
        assert np.array_equal(o["h"], whole["h"][c])
        assert np.array_equal(o["nsub"], whole["nsub"][c])
        assert np.array_equal(o["status"], whole["status"][c])
