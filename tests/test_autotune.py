"""Autotuner host logic (sample selection, search space, cache) on CPU, and on the GPU: a tuned launch
shape is one of the candidates, and every launch shape gives bit-identical results."""
import json

import numpy as np
import pytest

from paper_2311_14941_gb300 import autotune, synth


def test_sample_keeps_the_cost_distribution():
    rng = np.random.default_rng(1)
    cost = np.maximum(1, rng.lognormal(4, 1.2, 100000)).astype(np.int64)
    idx = autotune.sample_cells(len(cost), cost, 4096)
    assert len(idx) <= 4096 and len(idx) > 4000 and np.all(np.diff(idx) > 0)
    qs = [0.1, 0.5, 0.9, 0.99]
    assert np.allclose(np.quantile(cost[idx], qs), np.quantile(cost, qs), rtol=0.05)
    assert cost[idx].max() == cost.max()


def test_sample_without_counts_is_seeded_random_and_small_fields_are_whole():
    a = autotune.sample_cells(50000, None, 1000)
    b = autotune.sample_cells(50000, np.zeros(50000, np.int32), 1000)
    assert np.array_equal(a, b) and len(a) == 1000
    assert np.array_equal(autotune.sample_cells(500, None, 1000), np.arange(500))


def test_search_space():
    c = autotune.candidates({(1, 1): 7, (2, 1): 3, (1, 2): 13})
    assert {x["mode"] for x in c} == {0, 1} and {x["warps_per_cell"] for x in c} == {1, 2}
    one = [x for x in c if x["warps_per_cell"] == 1 and x["cells_per_warp"] == 1]
    assert {x["block_cells"] for x in one} == {1, 2, 4, 7}
    assert {x["block_cells"] for x in c if x["warps_per_cell"] == 2} == {1, 2, 3}
    # half-warp cells: whole warps only
    assert {x["block_cells"] for x in c if x["cells_per_warp"] == 2} == {2, 4, 8, 12}
    assert all(x["chunk"] == 1 for x in c if x["mode"] == 0)
    assert len({json.dumps(x, sort_keys=True) for x in c}) == len(c)
    assert {x["block_cells"] for x in autotune.candidates({(1, 1): 1})} == {1}


def test_block_bounds():
    # 24.6 KB cells in 227 KB: 9 per block; two-warp cells are also capped by 15 named barriers and 1024
    # threads
    assert autotune.max_block_cells(24592, 232448, 1) == 9
    assert autotune.max_block_cells(3616, 232448, 1) == 16
    assert autotune.max_block_cells(3616, 232448, 2) == 15
    assert autotune.max_block_cells(71048, 232448, 2) == 3


def test_digest_depends_on_every_parameter():
    m = synth.mechanism_small()
    d0 = autotune.mechanism_digest(m)
    assert d0 == autotune.mechanism_digest(synth.mechanism_small())
    m.Ea[3] *= 1.0000001
    assert autotune.mechanism_digest(m) != d0


def test_cache_roundtrip(tmp_path, monkeypatch):
    monkeypatch.setattr(autotune, "CACHE", str(tmp_path / "c.json"))
    assert autotune._load() == {}
    autotune._store("k1", {"warps_per_cell": 2, "mode": 1, "block_cells": 2, "chunk": 1})
    autotune._store("k2", {"warps_per_cell": 1, "mode": 0, "block_cells": 1, "chunk": 1})
    got = autotune._load()
    assert got["k1"]["block_cells"] == 2 and got["k2"]["mode"] == 0
    assert autotune.launch_options(got["k1"]) == {"warps_per_cell": 2, "cells_per_warp": 1, "mode": 1,
                                                  "block_cells": 2, "chunk": 1}


@pytest.mark.gpu
def test_gpu_launch_shapes_agree_and_tune_picks_one(tmp_path, monkeypatch):
    """Within one warps-per-cell choice every launch shape gives bit-identical results (a cell's arithmetic
    does not depend on where or when it runs); the two choices agree to rounding."""
    import torch
    from paper_2311_14941_gb300 import chem
    monkeypatch.setattr(autotune, "CACHE", str(tmp_path / "c.json"))
    m = synth.mechanism_methane_sized()
    F = synth.field_bimodal_jet(m, 48, 48, seed=3)
    h = chem.create(m, 0)
    dev = torch.device("cuda:0")
    t = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)
    N = F.n_cells
    ns_prev = torch.tensor(np.random.default_rng(2).integers(1, 300, N).astype(np.int32), device=dev)
    space = autotune.candidates({g: h.info["max_block_cells"][i] for i, g in enumerate(autotune.GROUPS)})
    optin = torch.cuda.get_device_properties(0).shared_memory_per_block_optin
    assert all(h.info["max_block_cells"][w - 1] <= autotune.max_block_cells(h.info["smem_per_cell"], optin, w)
               for w in (1, 2))
    assert h.info["auto_warps_per_cell"] == 1 and h.info["resident_cells"][0] >= 8
    ref = {}
    for c in space:
        T, Y = t(F.T), t(F.Y.reshape(-1))
        hio = torch.zeros(N, dtype=torch.float64, device=dev)
        ns = ns_prev.clone()
        st = torch.zeros(N, dtype=torch.int32, device=dev)
        h.integrate(T, t(F.p), Y, t(F.dt), hio, ns, st, **c)
        out = (T.cpu().numpy(), Y.cpu().numpy(), hio.cpu().numpy(), ns.cpu().numpy(), st.cpu().numpy())
        w = (c["warps_per_cell"], c["cells_per_warp"])
        if w not in ref:
            ref[w] = out
        for a, b in zip(out, ref[w]):
            assert np.array_equal(a, b), c
    a = ref[(1, 1)]
    big = np.abs(a[1]) > 1e-12
    for g in ((2, 1), (1, 2)):
        b = ref[g]
        assert np.all(a[4] == 0) and np.array_equal(a[4], b[4])
        assert np.allclose(a[0], b[0], rtol=1e-6, atol=0)
        assert np.allclose(a[1][big], b[1][big], rtol=1e-5, atol=0)
    r = autotune.tune(h, t(F.T), t(F.p), t(F.Y.reshape(-1)), t(F.dt), ns_prev, sample=1024)
    opts = autotune.launch_options(r)
    assert opts in [dict((k, x[k]) for k in autotune.KEYS) for x in space] or opts["block_cells"] == 0
    assert r["ms"] == min(x["ms"] for x in r["table"]) and r["ms"] > 0
    assert autotune.tune(h, t(F.T), t(F.p), t(F.Y.reshape(-1)), t(F.dt), ns_prev, sample=1024) == \
        json.loads(json.dumps(r))
