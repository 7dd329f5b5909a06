"""Launch-shape autotuner for chem_integrate.

Knobs searched:
  lane group      (warps_per_cell, cells_per_warp): (1, 1) one warp integrates a cell; (2, 1) two warps of
                  a block share it (wider reaction and species loops and twice the warps in flight, at the
                  price of more, emptier steps in the sparse factorisation and solves and of named-barrier
                  synchronisation); (1, 2) two cells share a warp, 16 lanes each (mechanisms with few
                  species, whose loops and sparse programs leave most of a warp idle)
  mode            0 = one grid over all cells, 1 = cells sorted by their previous substep count and
                  pulled by resident lane groups from an atomic queue (the on-chip form of the paper's
                  dynamic load balancing, Sec. 2.5)
  block_cells     cells per block: changes how shared memory is carved up per SM and how many blocks
                  share an SM
  chunk           cells a group claims per queue operation (mode 1)

The search is staged (coordinate descent): the lane group with the library's default block shape and
the sorted queue; then cells per block and queue chunk for that choice; then the plain grid with the
best block shape against the best queue.  Every run integrates the same sample of the caller's cells,
starting from the same state, once untimed and then timed with CUDA events on the caller's stream.  The
sample keeps the cost distribution of the whole field: cells are ordered by previous substep count and
every k-th is taken (a seeded random pick when no counts are known yet).  Results are cached per
(mechanism digest, cell-count bucket, device name, tolerances) in a JSON file next to the compiled
library.
"""
from __future__ import annotations

import hashlib
import json
import os

import numpy as np

from . import build as _build

CACHE = os.path.join(_build.OUT, "autotune_cache.json")
KEYS = ("warps_per_cell", "cells_per_warp", "mode", "block_cells", "chunk")
GROUPS = ((1, 1), (2, 1), (1, 2))   # (warps_per_cell, cells_per_warp), in the order of chem_info's arrays


def mechanism_digest(desc) -> str:
    h = hashlib.sha1()
    for name in ("W", "nasa_lo", "nasa_hi", "T_mid", "reac_ptr", "reac_sp", "reac_nu", "prod_ptr", "prod_sp",
                 "prod_nu", "A", "b", "Ea", "rtype", "reversible", "eff_ptr", "eff_sp", "eff_alpha", "troe", "low"):
        h.update(np.ascontiguousarray(getattr(desc, name)).tobytes())
    return h.hexdigest()[:16]


def max_block_cells(cell_bytes: int, smem_optin: int, warps_per_cell: int) -> int:
    """Most cells a block can hold by shared memory, 1024 threads, at most 16, and 15 named barriers for
    two-warp cells (the library also applies the kernels' register limit: chem_info max_block_cells)."""
    c = max(1, smem_optin // max(cell_bytes, 1))
    c = min(c, 1024 // (32 * warps_per_cell), 16)
    if warps_per_cell > 1:
        c = min(c, 15)
    return max(1, c)


def block_shapes(max_cells: int, cells_per_warp: int = 1):
    if cells_per_warp == 2:   # half-warp cells come in pairs (whole warps)
        return sorted({c for c in (2, 4, 8, max_cells - max_cells % 2) if 2 <= c <= max_cells})
    return sorted({c for c in (1, 2, 4, max_cells) if c <= max_cells})


def candidates(max_cells: dict):
    """The full launch-shape space; max_cells[g] = largest block (in cells) for lane group g = (warps per
    cell, cells per warp)."""
    out = []
    for g in sorted(max_cells):
        wpc, cpw = g
        shapes = block_shapes(max_cells[g], cpw)
        out += [dict(warps_per_cell=wpc, cells_per_warp=cpw, mode=0, block_cells=c, chunk=1) for c in shapes]
        out += [dict(warps_per_cell=wpc, cells_per_warp=cpw, mode=1, block_cells=c, chunk=k) for c in shapes
                for k in (1, 2, 4)]
    return out


def sample_cells(n_cells: int, nsub_prev=None, size: int = 8192, seed: int = 0) -> np.ndarray:
    """Indices of a cost-stratified sample of at most `size` cells."""
    if n_cells <= size:
        return np.arange(n_cells)
    if nsub_prev is None or not np.any(np.asarray(nsub_prev)):
        return np.sort(np.random.default_rng(seed).choice(n_cells, size, replace=False))
    order = np.argsort(-np.asarray(nsub_prev), kind="stable")
    pick = order[np.linspace(0, n_cells - 1, size).round().astype(np.int64)]
    return np.sort(np.unique(pick))


def _key(mech, n_cells, rtol, atol):
    import torch
    bucket = 1 << max(0, int(np.ceil(np.log2(max(n_cells, 1)))))
    dev = torch.cuda.get_device_name(mech.device)
    return f"{mechanism_digest(mech.desc)}|{bucket}|{dev}|{rtol:g}|{atol:g}"


def _load():
    try:
        with open(CACHE) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(key, value):
    data = _load()
    data[key] = value
    os.makedirs(os.path.dirname(CACHE), exist_ok=True)
    tmp = CACHE + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, CACHE)


def tune(mech, T, p, Y, dt, nsub_prev=None, rtol=1e-6, atol=1e-12, sample: int = 8192, use_cache: bool = True,
         repeats: int = 1, stream=None):
    """Best launch shape for integrating these cells; returns {warps_per_cell, cells_per_warp, mode,
    block_cells, chunk, ms, sample, table}.

    T, p, dt: device tensors [N]; Y: [n*N] species-major; nsub_prev: previous substep counts (device or
    host, may be None).  The inputs are not modified."""
    import torch
    N = T.numel()
    key = _key(mech, N, rtol, atol)
    if use_cache:
        hit = _load().get(key)
        if hit is not None:
            return hit
    ns_host = None if nsub_prev is None else np.asarray(
        nsub_prev.cpu().numpy() if hasattr(nsub_prev, "cpu") else nsub_prev)
    idx = sample_cells(N, ns_host, sample)
    ii = torch.as_tensor(idx, device=T.device)
    n = mech.n
    Ts, Ps, Ds = T[ii].contiguous(), p[ii].contiguous(), dt[ii].contiguous()
    Ys = Y.view(n, N)[:, ii].contiguous().view(-1)
    ns0 = torch.zeros(len(idx), dtype=torch.int32, device=T.device) if ns_host is None else \
        torch.as_tensor(ns_host[idx].astype(np.int32), device=T.device)
    info = mech.info
    maxc = {g: int(info["max_block_cells"][i]) for i, g in enumerate(GROUPS)}
    strm = stream or torch.cuda.current_stream(T.device)
    Tw, Yw = torch.empty_like(Ts), torch.empty_like(Ys)
    hio = torch.empty(len(idx), dtype=torch.float64, device=T.device)
    ns = torch.empty_like(ns0)
    st = torch.empty_like(ns0)
    table = []

    def timed(c):
        times = []
        for r in range(1 + repeats):
            with torch.cuda.stream(strm):
                Tw.copy_(Ts)
                Yw.copy_(Ys)
                hio.zero_()
                ns.copy_(ns0)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(strm)
                mech.integrate(Tw, Ps, Yw, Ds, hio, ns, st, rtol=rtol, atol=atol, stream=strm, **c)
                e1.record(strm)
            strm.synchronize()
            if r > 0:
                times.append(e0.elapsed_time(e1))
        row = dict(c, ms=float(min(times)))
        table.append(row)
        return row

    # 1) lane group, library default block shape, sorted queue
    best = min((timed(dict(warps_per_cell=w, cells_per_warp=cpw, mode=1, block_cells=0, chunk=1))
                for w, cpw in GROUPS), key=lambda d: d["ms"])
    w, cpw = best["warps_per_cell"], best["cells_per_warp"]
    # 2) block shape and chunk for that choice
    for c in block_shapes(maxc[(w, cpw)], cpw):
        for k in (1, 2, 4):
            row = timed(dict(warps_per_cell=w, cells_per_warp=cpw, mode=1, block_cells=c, chunk=k))
            if row["ms"] < best["ms"]:
                best = row
    # 3) the plain grid with that block shape
    row = timed(dict(warps_per_cell=w, cells_per_warp=cpw, mode=0, block_cells=best["block_cells"], chunk=1))
    if row["ms"] < best["ms"]:
        best = row
    out = dict({k: best[k] for k in KEYS}, ms=best["ms"], sample=int(len(idx)), table=table)
    if use_cache:
        _store(key, out)
    return out


def launch_options(result) -> dict:
    """The chem_integrate keyword arguments of a `tune` result (results cached before the lane-group
    choice existed mean one cell per warp)."""
    return {k: int(result.get(k, 1)) for k in KEYS}
