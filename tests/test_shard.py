"""Cell sharding over ranks: the cost-balanced partition, and a two-rank gloo run on CPU of the
multi-rank path (partition agreed without communication, independent per-rank integration,
gradient all-reduce, max-over-ranks timing)."""
import os
import socket

import numpy as np
import pytest

from paper_2311_14941_gb300 import shard


@pytest.mark.parametrize("world", [1, 2, 3, 4, 7])
def test_partition_covers_every_cell_once(world):
    cost = np.random.default_rng(world).integers(1, 5000, 1001)
    parts = shard.partition(cost, world)
    assert len(parts) == world
    allc = np.concatenate(parts)
    assert np.array_equal(np.sort(allc), np.arange(len(cost)))
    for p in parts:
        assert np.all(np.diff(p) > 0)


def test_partition_balances_heavy_tailed_cost():
    rng = np.random.default_rng(3)
    cost = np.maximum(1, rng.lognormal(4.0, 1.5, 20000)).astype(np.int64)
    for world in (2, 4, 8):
        sums = np.array([cost[p].sum() for p in shard.partition(cost, world)])
        # greedy least-loaded assignment in descending cost bounds the spread by the largest single cost
        assert sums.max() - sums.min() <= cost.max()
        assert sums.max() / sums.mean() < 1.001


def test_partition_equal_costs_deal_evenly():
    parts = shard.partition(np.ones(10), 4)
    assert sorted(len(p) for p in parts) == [2, 2, 3, 3]


def test_partition_is_deterministic_with_ties():
    cost = np.array([5, 5, 5, 1, 1, 9, 9, 0])
    a = shard.partition(cost, 3)
    b = shard.partition(cost.copy(), 3)
    assert all(np.array_equal(x, y) for x, y in zip(a, b))
    with pytest.raises(ValueError):
        shard.partition(cost, 0)
    with pytest.raises(ValueError):
        shard.local_cells(cost, 3, 3)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, outdir):
    import torch
    import torch.distributed as dist
    from oracle.oracle import Oracle
    from paper_2311_14941_gb300 import synth
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        m = synth.mechanism_small()
        F = synth.field_uniform_random(m, 24, seed=5)
        cost = np.random.default_rng(9).integers(1, 400, F.n_cells)     # previous substep counts
        mine = shard.local_cells(cost, rank, world)
        S = F.subset(mine)
        r = Oracle(m).integrate_batch(S.T, S.p, S.Y, S.dt, 1e-6, 1e-12, nthreads=1)
        # the per-rank parameter gradients: stand-in values that depend on the rank
        gA = torch.arange(5, dtype=torch.float64) * (rank + 1)
        gE = torch.full((5,), 10.0 ** rank, dtype=torch.float64)
        shard.allreduce_gradients(gA, gE)
        tmax = shard.max_over_ranks(0.5 + rank)
        np.savez(os.path.join(outdir, f"r{rank}.npz"), cells=mine, T=r["T"], Y=r["Y"], gA=gA.numpy(),
                 gE=gE.numpy(), tmax=tmax)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_integrate_disjoint_shards(tmp_path):
    import torch.multiprocessing as mp
    from oracle.oracle import Oracle
    from paper_2311_14941_gb300 import synth
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, start_method="spawn",
                       join=True)
    out = [np.load(tmp_path / f"r{r}.npz") for r in range(world)]
    cells = np.concatenate([o["cells"] for o in out])
    assert np.array_equal(np.sort(cells), np.arange(24))
    # sharded results are the unsharded ones: no data-path exchange is needed
    m = synth.mechanism_small()
    F = synth.field_uniform_random(m, 24, seed=5)
    whole = Oracle(m).integrate_batch(F.T, F.p, F.Y, F.dt, 1e-6, 1e-12, nthreads=1)
    for o in out:
        c = o["cells"]
        assert np.array_equal(o["T"], whole["T"][c])
        assert np.array_equal(o["Y"], whole["Y"][:, c])
    for o in out:
        assert np.array_equal(o["gA"], np.arange(5) * 3.0)
        assert np.array_equal(o["gE"], np.full(5, 11.0))
        assert float(o["tmax"]) == 1.5
