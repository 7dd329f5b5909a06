"""Benchmark: reactor-steps/s of the stiff chemistry integrator on GB300.

One step = one chem_integrate call advancing every cell of the workload over its flow time step dt
(a "reactor-step" is one cell integrated over its dt).  Workloads (--workload):
  lts    (default) 53-species / 325-reaction synthetic mechanism on 262,144 cells (70 % cold 300-600 K,
         20 % burnt 1600-2200 K, 10 % igniting 1000-1300 K) with per-cell dt log-uniform in
         [1e-7, 1e-3] s.  The field evolves over episodes of 10 consecutive flow steps: each episode
         starts from the initial field with no substep history, its step 1 (untimed) seeds the substep
         counts that the sorted queue uses as its cost key, and its steps 2-10 are timed; the timed steps
         run through as many episodes as --steps needs.  The persistent sorted queue is the headline and
         the plain grid is timed on the first episode's steps 2-10 beside it (the same states: the two
         launches give bit-identical results).
  jet    the same mechanism on the 65,536-cell bimodal jet field (40 % unburnt, 60 % burnt, mixing
         layer), uniform dt = 1e-5 s; every step starts from the same initial state (restored by device
         copies inside the step); also reported as a secondary key of the lts line
  large  150-species / 1000-reaction mechanism on a 131,072-cell bimodal field, per-cell dt log-uniform
         in [1e-6, 1e-4] s, state restored every step
FP64, rtol 1e-6 / atol 1e-12.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--workload lts|jet|large] [--impl reference]
Prints one JSON line (rank 0).  With torchrun each rank integrates its own field (weak scaling).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "reactor-steps/s, 53sp/325rxn FP64 rtol1e-6: persistent vs plain; adjoint s/grad"
RTOL, ATOL = 1e-6, 1e-12
METHODS = {"rodas3": 0, "ros2": 1, "rodas4": 2}   # chem_integrate_opts.method

# DRAM bytes per cell of the integration kernel, from one ncu capture of 32,768 cells of the LTS field
# (dram__bytes_read.sum + dram__bytes_write.sum = 16.40 MB, episode step 2; the traffic scales with the
# cell count: the state is read once, tables are L2-resident, the written state stays in L2).  Valid
# only for the kernel sources it was taken on: the digest below is checked at run time and the traffic
# is reported as null after any change.
PROFILED_TRAFFIC_PER_CELL = {"lts": (15897600 + 504832) / 32768}
PROFILED_SOURCES = "e471941195af2a5c"
REF_CELLS = 256   # reference arm: cells per step (at least 16 per host core)
KERNEL_SOURCES = ["integrate.cuh", "kern_forward.cuh", "kern_fwd_warp.cu", "kernels.cuh", "compile.cpp", "device.cuh",
                  "elementary_tables.h", "mech.h", "scalar.cuh"]


def kernel_sources_digest():
    import hashlib
    h = hashlib.sha1()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2311_14941_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]

WORKLOADS = {
    "jet": {"workload": "methane-sized 53sp/325rxn, 65536-cell bimodal jet field (40% unburnt 300-600 K, "
                        "60% burnt 1600-2200 K, tanh mixing layer), uniform dt=1e-5 s",
            "n_cells": 65536, "evolving": False},
    "lts": {"workload": "methane-sized 53sp/325rxn, 262144-cell LTS mix (70% cold 300-600 K, 20% burnt "
                        "1600-2200 K, 10% igniting 1000-1300 K), per-cell dt log-uniform 1e-7..1e-3 s, "
                        "evolving field in episodes of 10 flow steps (step 1 seeds the sort key, steps 2-10 "
                        "timed)",
            "n_cells": 262144, "evolving": True},
    "large": {"workload": "large 150sp/1000rxn, 131072-cell bimodal jet field (512x256), per-cell dt "
                          "log-uniform 1e-6..1e-4 s",
              "n_cells": 131072, "evolving": False},
    "small": {"workload": "small 10sp/27rxn (H, O, N), 1024 cells, p = 1 atm, T uniform 900-2200 K, Dirichlet Y, "
                          "dt=1e-5 s",
              "n_cells": 1024, "evolving": False},
    "small64k": {"workload": "small 10sp/27rxn (H, O, N), 65536 cells drawn like the 1024-cell case (p = 1 atm, "
                             "T uniform 900-2200 K, Dirichlet Y, dt=1e-5 s)",
                 "n_cells": 65536, "evolving": False},
}


EPISODE = 10   # flow steps per episode of an evolving workload; step 1 of each is untimed


def workload(name="lts", seed_offset=0):
    from paper_2311_14941_gb300 import synth
    if name == "jet":
        m = synth.mechanism_methane_sized()
        F = synth.field_bimodal_jet(m, 256, 256, seed=2 + seed_offset, dt=1e-5)
    elif name == "lts":
        m = synth.mechanism_methane_sized()
        F = synth.field_lts_mix(m, 262144, seed=3 + seed_offset)
    elif name == "large":
        m = synth.mechanism_large()
        F = synth.field_bimodal_jet(m, 512, 256, seed=5 + seed_offset, dt_range=(1e-6, 1e-4))
    elif name in ("small", "small64k"):
        m = synth.mechanism_small()
        F = synth.field_uniform_random(m, WORKLOADS[name]["n_cells"], seed=1 + seed_offset)
    else:
        raise ValueError(name)
    return m, F


def config(name, mode):
    w = WORKLOADS[name]
    c = {"workload": w["workload"], "n_cells": w["n_cells"], "rtol": RTOL, "atol": ATOL, "mode": mode,
         "l2": "flushed between timed steps (256 MiB write)"}
    c["state"] = (f"advanced from step to step in episodes of {EPISODE} flow steps from the initial field; "
                  "step 1 of each episode seeds the substep counts and is not timed" if w["evolving"]
                  else "restored to the same initial field each step")
    return c


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, path):
        self.path = path
        self.proc = None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.f.close()

    def summary(self, device_index=0):
        if self.proc is None or not os.path.exists(self.path):
            return None
        sm, mx, reasons = [], None, set()
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                if int(parts[0]) != device_index:
                    continue
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def cpu_baseline(m, F, name, budget_s=12.0, method=0):
    """The oracle as it stands on this host's cores over a bounded sample of the workload's cells, with the
    same Rosenbrock method and tolerances as the timed GPU run."""
    from oracle.oracle import Oracle
    o = Oracle(m)
    rng = np.random.default_rng(11)
    idx = rng.permutation(F.n_cells)
    done, t_used, chunk = 0, 0.0, 64
    threads = 0
    while t_used < budget_s and done < F.n_cells:
        sl = idx[done:done + chunk]
        S = F.subset(sl)
        t0 = time.perf_counter()
        r = o.integrate_batch(S.T, S.p, S.Y, S.dt, RTOL, ATOL, method=method)
        t_used += time.perf_counter() - t0
        threads = r["threads"]
        done += len(sl)
        chunk = min(chunk * 2, 1024)
    # the same oracle on one core, over the first cells of the same sample
    one, t_one = 0, 0.0
    while t_one < budget_s / 2 and one < F.n_cells:
        sl = idx[one:one + 8]
        S = F.subset(sl)
        t0 = time.perf_counter()
        o.integrate_batch(S.T, S.p, S.Y, S.dt, RTOL, ATOL, method=method, nthreads=1)
        t_one += time.perf_counter() - t0
        one += len(sl)
    return {"value": done / t_used, "unit": "reactor-steps/s", "cores": int(threads), "kind": "oracle",
            "sample": f"{done} seeded-random cells of the {name} workload's initial field, each integrated over "
                      f"its dt with OpenMP over cells ({t_used:.1f} s)",
            "single_core": {"value": one / t_one, "unit": "reactor-steps/s", "cores": 1,
                            "sample": f"the first {one} cells of the same sample ({t_one:.1f} s)"}}


def adjoint_fields(name, m, F):
    """Adjoint workload: 4096 igniting cells to t = 1e-3 s for the 53/325 mechanism; a seeded 2048-cell
    subset of the field for the 150/1000 one."""
    from paper_2311_14941_gb300 import synth
    rank = int(os.environ.get("RANK", "0"))
    if name == "large":
        idx = np.sort(np.random.default_rng(21 + rank).choice(F.n_cells, 2048, replace=False))
        return F.subset(idx), "150sp/1000rxn, seeded 2048-cell subset of the bimodal field, own dt"
    return (synth.field_igniting(m, 4096, seed=4 + rank, dt=1e-3),
            "53sp/325rxn igniting cells, T0 1000-1400 K, p 1-10 atm, integrated to 1e-3 s")


def adjoint_bench(h, m, dev, F, label):
    """Seconds per gradient: one chem_adjoint call (one cotangent vector, all cells, all 2R parameters);
    objective = final T (x1e-3) plus 5 seeded species mass fractions; checkpoints every 16 accepted
    steps.  The forward integration of the same cells is timed alone for the cost ratio."""
    import torch
    from paper_2311_14941_gb300 import shard, synth
    sel = synth.cotangent_species(m, 5, seed=4)
    t = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)
    N = F.n_cells
    gT = t(np.full(N, 1e-3))
    gYn = np.zeros((m.n_species, N))
    gYn[sel] = 1.0
    gY = t(gYn.reshape(-1))
    gA = torch.zeros(h.R, dtype=torch.float64, device=dev)
    gE = torch.zeros(h.R, dtype=torch.float64, device=dev)
    st = torch.zeros(N, dtype=torch.int32, device=dev)
    P, D = t(F.p), t(F.dt)
    # untimed call on all cells over a 1e-12 s interval: loads the module and sizes the scratch (it
    # depends on the cell count and the tape options only)
    T, Y = t(F.T), t(F.Y.reshape(-1))
    h.adjoint(T, P, Y, torch.full_like(D, 1e-12), gT, gY, gA, gE, st)
    torch.cuda.synchronize()
    T, Y = t(F.T), t(F.Y.reshape(-1))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    h.adjoint(T, P, Y, D, gT, gY, gA, gE, st)
    shard.allreduce_gradients(gA, gE)      # ranks sum their cells' parameter gradients (no-op on one GPU)
    e1.record()
    torch.cuda.synchronize()
    s = shard.max_over_ranks(e0.elapsed_time(e1) / 1e3, dev)
    stat = st.cpu().numpy()
    T, Y = t(F.T), t(F.Y.reshape(-1))
    hio = torch.zeros(N, dtype=torch.float64, device=dev)
    ns = torch.zeros(N, dtype=torch.int32, device=dev)
    st2 = torch.zeros(N, dtype=torch.int32, device=dev)
    e0.record()
    h.integrate(T, P, Y, D, hio, ns, st2, rtol=RTOL, atol=ATOL, mode=0)
    e1.record()
    torch.cuda.synchronize()
    s_fwd = e0.elapsed_time(e1) / 1e3
    return {"s_per_grad": s, "forward_s": s_fwd, "cells": N, "params": 2 * h.R,
            "cotangent": "final T (x1e-3) + 5 seeded species", "workload": label + ", checkpoints every 16 "
            "accepted steps", "substeps_mean": float(ns.float().mean().item()),
            "cell_status": {str(k): int(v) for k, v in zip(*np.unique(stat, return_counts=True))},
            "grad_norm": float(torch.linalg.vector_norm(torch.cat([gA, gE])).item())}


def map_options(F, T_max):
    """Zonal mapping of the cells below T_max: 20 K temperature bins and 0.02 bins of the two mass
    fractions that vary most over those cells."""
    low = F.T < T_max
    sp = np.argsort(-F.Y[:, low].std(axis=1))[:2] if low.any() else np.arange(2)
    return {"T_max": float(T_max), "dT": 20.0, "species": [int(x) for x in sp], "dY": [0.02, 0.02]}


def mapped_bench(h, F, args, T0, Y0, P, DTs, T, Y, hio, ns, st, flush, stream, meth, world, dev):
    """The same steps through chem_integrate_mapped (each from the same initial field): cells advanced per
    second, counting mapped cells as advanced, and the mapping's deviation from the unmapped result that
    T and Y hold on entry."""
    import torch
    from paper_2311_14941_gb300 import shard
    N = F.n_cells
    mp = map_options(F, args.map_tmax)
    ref = torch.empty(N, dtype=torch.int32, device=dev)
    Tu, Yu = T.clone(), Y.clone()
    mode = 1 if args.mode == "persistent" else 0

    def step():
        T.copy_(T0)
        Y.copy_(Y0)
        hio.zero_()
        return h.integrate_mapped(T, P, Y, DTs, hio, ns, st, ref, mp, rtol=RTOL, atol=ATOL, mode=mode, method=meth)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    M = 0
    for i in range(args.steps):
        flush.fill_(float(i))
        evs[i][0].record(stream)
        M = step()
        evs[i][1].record(stream)
    torch.cuda.synchronize()
    t = shard.max_over_ranks(sum(a.elapsed_time(b) for a, b in evs) / 1e3, dev)
    n = F.Y.shape[0]
    return {"value": world * N * args.steps / t, "unit": "reactor-steps/s (mapped cells count as advanced)",
            "ms_per_step": 1e3 * t / args.steps, "integrated_cells": int(M), "mapping": mp,
            "max_abs_dT_vs_unmapped": float((T - Tu).abs().max()),
            "max_abs_dY_vs_unmapped": float((Y - Yu).view(n, N).abs().max()),
            "status": {str(k): int(v) for k, v in zip(*np.unique(st.cpu().numpy(), return_counts=True))}}


def run_reference(args):
    """The reference arm: the oracle as it stands on this host's cores, on samples of the same workload with
    the same metric, method and tolerances.  Each step integrates REF_CELLS seeded-random cells of the
    workload's initial field (dt descending, so the long cells start first), enough for every core."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    m, F = workload(args.workload)
    from oracle.oracle import Oracle
    o = Oracle(m)
    rng = np.random.default_rng(13)
    per_step = max(REF_CELLS, 16 * (os.cpu_count() or 1))
    meth = METHODS[args.method]

    def sample():
        idx = rng.choice(F.n_cells, per_step, replace=False)
        return F.subset(idx[np.argsort(-F.dt[idx], kind="stable")])

    for _ in range(args.warmup):
        S = sample()
        o.integrate_batch(S.T, S.p, S.Y, S.dt, RTOL, ATOL, method=meth)
    t, threads = 0.0, 0
    for _ in range(args.steps):
        S = sample()
        t0 = time.perf_counter()
        r = o.integrate_batch(S.T, S.p, S.Y, S.dt, RTOL, ATOL, method=meth)
        t += time.perf_counter() - t0
        threads = r["threads"]
    v = per_step * args.steps / t
    smp = (f"{per_step} seeded-random cells of the workload's initial field per step (no substep history), "
           f"OpenMP over cells one at a time on {threads} threads")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "reactor-steps/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": dict(config(args.workload, "oracle"), sample=smp, method=args.method),
            "cpu_baseline": {"value": v, "unit": "reactor-steps/s", "cores": threads, "kind": "oracle",
                             "sample": smp},
            "e2e": {"value": v, "unit": "reactor-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


class Runner:
    """Timed chem_integrate steps on one workload: buffers, the step schedule and the work counts."""

    def __init__(self, h, F, evolving, dev, meth, oc, world, flush, clocks_path, local, cells_per_warp=0,
                 tab_tol=0.0, specialized=0):
        import torch
        self.h, self.F, self.evolving, self.dev, self.meth, self.oc = h, F, evolving, dev, meth, oc
        self.cpw = cells_per_warp
        self.spec = specialized
        self.tab = dict(tabulate=1, tab_tol=tab_tol) if tab_tol > 0 else {}
        self.world, self.flush, self.clocks_path, self.local = world, flush, clocks_path, local
        N = F.n_cells
        self.N = N
        self.T0 = torch.tensor(F.T, device=dev)
        self.Y0 = torch.tensor(F.Y.reshape(-1), device=dev)
        self.P = torch.tensor(F.p, device=dev)
        self.DT = torch.tensor(F.dt, device=dev)
        self.T = torch.empty_like(self.T0)
        self.Y = torch.empty_like(self.Y0)
        self.hio = torch.zeros(N, dtype=torch.float64, device=dev)
        self.ns = torch.zeros(N, dtype=torch.int32, device=dev)
        self.st = torch.zeros(N, dtype=torch.int32, device=dev)
        self.nacc = torch.zeros(N, dtype=torch.int32, device=dev)
        self.stream = torch.cuda.current_stream()
        self.k = 0   # flow step within the current episode (evolving workloads)

    def reset(self):
        """Initial field, no step-size or substep history."""
        self.T.copy_(self.T0)
        self.Y.copy_(self.Y0)
        self.hio.zero_()
        self.ns.zero_()
        self.k = 0

    def integrate(self, mode):
        self.h.integrate(self.T, self.P, self.Y, self.DT, self.hio, self.ns, self.st, rtol=RTOL, atol=ATOL,
                         mode=mode, naccept=self.nacc, method=self.meth, cells_per_warp=self.cpw,
                         specialized=self.spec, **self.tab)

    def step(self, mode):
        """One flow step.  Evolving: the next step of the episode.  Otherwise: from the initial state again,
        with the previous call's substep counts as the sort key."""
        if self.evolving:
            self.integrate(mode)
            self.k += 1
        else:
            self.T.copy_(self.T0)
            self.Y.copy_(self.Y0)
            self.hio.zero_()
            self.integrate(mode)

    def ready_for_timed_step(self, mode):
        """Evolving workloads: start a new episode (reset and its untimed seeding step) when the current one
        is used up or has not begun.  Runs outside the timed events."""
        if self.evolving and (self.k == 0 or self.k >= EPISODE):
            self.reset()
            self.step(mode)

    def run(self, mode_name, n_warm, n_timed, count_work=True):
        """n_warm untimed steps, then n_timed timed steps (CUDA events on the launching stream, L2 flushed
        before each).  Evolving workloads start the timed steps from a fresh episode."""
        import torch
        import torch.distributed as dist
        from paper_2311_14941_gb300 import shard
        mode = 1 if mode_name == "persistent" else 0
        self.reset()
        for _ in range(n_warm):
            if self.evolving and self.k >= EPISODE:
                self.reset()
            self.step(mode)
        torch.cuda.synchronize()
        if self.evolving:
            self.k = 0
        else:   # the sort key of the first timed step: the counts of a full step from the same state
            self.step(mode)
        if self.world > 1:
            dist.barrier()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n_timed)]
        slots, subs = 0.0, 0
        ep_steps = []
        torch.cuda.synchronize()
        with Clocks(self.clocks_path) as ck:
            for i in range(n_timed):
                self.ready_for_timed_step(mode)
                ep_steps.append(self.k + 1)
                self.flush.fill_(float(i))
                evs[i][0].record(self.stream)
                self.step(mode)
                evs[i][1].record(self.stream)
                if count_work and (self.evolving or i == 0):   # per-step work (outside the timed events)
                    ns_h = self.ns.cpu().numpy()
                    slots += float(self.oc.cell_slots(ns_h, self.nacc.cpu().numpy()).sum())
                    subs += int(ns_h.sum())
            torch.cuda.synchronize()
        if self.world > 1:
            dist.barrier()
        step_ms = [a.elapsed_time(b) for a, b in evs]
        if not self.evolving:   # every step repeats the same work
            slots *= n_timed
            subs *= n_timed
        t_total = shard.max_over_ranks(sum(step_ms) / 1e3, self.dev)
        if self.world > 1:   # substeps of the whole job
            tot = torch.tensor([float(subs)], dtype=torch.float64, device=self.dev)
            dist.all_reduce(tot)
            subs = int(tot.item())
        return {"t": t_total, "step_ms": step_ms, "slots": slots, "subs": subs, "nsub": self.ns.cpu().numpy(),
                "nacc": self.nacc.cpu().numpy(), "status": self.st.cpu().numpy(), "clocks": ck.summary(self.local),
                "episode_steps": ep_steps if self.evolving else None}

    def e2e(self, mode, n_steps):
        """End to end through the ABI with pinned host buffers: every step uploads the state (T, Y, h, nsub)
        and the cell data (p, dt), integrates and downloads the state and the status.  Evolving workloads
        start from the seeded step 1 of an episode and carry the state through the host."""
        import torch
        from paper_2311_14941_gb300 import shard
        N = self.N
        self.reset()
        self.step(mode)   # evolving: the episode's seeding step 1; otherwise a full step for the sort key
        if not self.evolving:
            self.hio.zero_()
        torch.cuda.synchronize()
        Th, Yh, Hh, Nh = (x.cpu().pin_memory() for x in ((self.T, self.Y) if self.evolving else (self.T0, self.Y0))
                          + (self.hio, self.ns))
        Ph, Dh = self.P.cpu().pin_memory(), self.DT.cpu().pin_memory()
        To, Yo, Ho, No = (torch.empty_like(x).pin_memory() for x in (Th, Yh, Hh, Nh))
        So = torch.empty(N, dtype=torch.int32).pin_memory()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(n_steps):
            self.T.copy_(Th, non_blocking=True)
            self.Y.copy_(Yh, non_blocking=True)
            self.hio.copy_(Hh, non_blocking=True)
            self.ns.copy_(Nh, non_blocking=True)
            self.P.copy_(Ph, non_blocking=True)
            self.DT.copy_(Dh, non_blocking=True)
            self.h.integrate(self.T, self.P, self.Y, self.DT, self.hio, self.ns, self.st, rtol=RTOL, atol=ATOL,
                             mode=mode, method=self.meth, cells_per_warp=self.cpw, specialized=self.spec,
                             **self.tab)
            To.copy_(self.T, non_blocking=True)
            Yo.copy_(self.Y, non_blocking=True)
            Ho.copy_(self.hio, non_blocking=True)
            No.copy_(self.ns, non_blocking=True)
            So.copy_(self.st, non_blocking=True)
            torch.cuda.synchronize()
            if self.evolving:
                Th, To, Yh, Yo, Hh, Ho = To, Th, Yo, Yh, Ho, Hh
            Nh, No = No, Nh
        t = shard.max_over_ranks(time.perf_counter() - t0, self.dev)
        h2d = sum(x.numel() * x.element_size() for x in (Th, Yh, Hh, Nh, Ph, Dh))
        d2h = sum(x.numel() * x.element_size() for x in (To, Yo, Ho, No, So))
        return {"value": self.world * N * n_steps / t, "unit": "reactor-steps/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "steps": n_steps}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=9)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default="lts", choices=sorted(WORKLOADS))
    ap.add_argument("--mode", default="persistent", choices=["plain", "persistent"],
                    help="the mode of the headline value (the other one is timed beside it)")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-other-mode", action="store_true", help="time only --mode")
    ap.add_argument("--no-secondary", action="store_true", help="skip the jet-field key of the lts line")
    ap.add_argument("--cells", type=int, default=0, help="integrate only this many seeded-random cells (profiling)")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the adjoint seconds-per-gradient measurement")
    ap.add_argument("--rtol", type=float, default=1e-6, help="relative tolerance (the headline metric is at 1e-6)")
    ap.add_argument("--map-tmax", type=float, default=0.0,
                    help="also time chem_integrate_mapped with cells below this temperature mapped (0: off)")
    ap.add_argument("--method", default="rodas3", choices=list(METHODS),
                    help="Rosenbrock method of the forward integration (the headline is RODAS3)")
    ap.add_argument("--cells-per-warp", type=int, default=0, choices=[0, 1, 2],
                    help="2: two cells share a warp (16 lanes each); 1: one cell per warp; 0: the library's choice")
    ap.add_argument("--tabulate", type=float, default=0.0,
                    help="evaluate the costly temperature functions from tables of this relative tolerance "
                         "(an approximation; 0: exact)")
    ap.add_argument("--kernels", default="auto", choices=["auto", "library", "specialized"],
                    help="integration kernels of the headline: the mechanism-specialised ones (run-time "
                         "compiled, one warp per cell), the library's, or auto = specialised where the "
                         "workload runs one cell per warp and the compile succeeds")
    ap.add_argument("--no-specialized-ab", action="store_true",
                    help="skip timing the other kernel build beside the headline's on the same steps")
    args = ap.parse_args()
    global RTOL
    RTOL = args.rtol
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import torch.distributed as dist
    from paper_2311_14941_gb300 import chem, opcount

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    m, F = workload(args.workload, seed_offset=rank)
    if args.cells:
        F = F.subset(np.sort(np.random.default_rng(5).permutation(F.n_cells)[: args.cells]))
    evolving = WORKLOADS[args.workload]["evolving"]
    meth = METHODS[args.method]
    h = chem.create(m, local)
    one_warp = (args.cells_per_warp or int(h.info["auto_cells_per_warp"])) == 1 and \
        int(h.info["auto_warps_per_cell"]) == 1
    spec_info = None
    if args.kernels == "specialized" or (one_warp and (args.kernels == "auto" or not args.no_specialized_ab)):
        try:   # compiled before any timing; the time is reported, not counted
            spec_info = {"compile_s": h.specialize()}
        except chem.ChemError as e:
            if args.kernels == "specialized":
                raise
            spec_info = {"unavailable": str(e)}
    args.specialized = args.kernels == "specialized" or (
        args.kernels == "auto" and one_warp and spec_info is not None and "compile_s" in spec_info)
    oc = opcount.model(m, h.export_plan(0), h.export_plan(1), method=meth)
    N = F.n_cells
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)   # 256 MiB > L2
    import tempfile
    clocks_path = os.path.join(tempfile.gettempdir(), f"chem_bench_clocks_r{rank}_{os.getpid()}.csv")
    run = Runner(h, F, evolving, dev, meth, oc, world, flush, clocks_path, local, args.cells_per_warp, args.tabulate,
                 1 if args.specialized else 0)

    # headline mode first (W warm-up, K timed), then the other mode on the first K' of the same steps:
    # for an evolving field, the first episode's steps 2-10 (bit-identical states in both modes)
    res = run.run(args.mode, args.warmup, args.steps)
    other = "plain" if args.mode == "persistent" else "persistent"
    res_other = None
    k_other = min(args.steps, EPISODE - 1) if evolving else args.steps
    if not args.no_other_mode:
        res_other = run.run(other, 1, k_other, count_work=False)
    # A/B of the kernels: the other build (specialised vs the library's) in the headline mode, same steps
    res_ab = None
    if spec_info is not None and "compile_s" in spec_info and one_warp and not args.no_specialized_ab:
        run.spec = 0 if args.specialized else 1
        res_ab = run.run(args.mode, 1, k_other, count_work=False)
        run.spec = 1 if args.specialized else 0
    t_total = res["t"]
    value = world * N * args.steps / t_total

    # roofline: algorithmic FP64 work of the launches / their duration
    achieved = opcount.FLOP_PER_SLOT * res["slots"] / t_total / 1e12
    peak = opcount.fp64_peak_tflops()
    traffic = None
    if kernel_sources_digest() == PROFILED_SOURCES and args.workload in PROFILED_TRAFFIC_PER_CELL:
        traffic = PROFILED_TRAFFIC_PER_CELL[args.workload] * N

    # end to end over the same flow steps as the first timed ones (an evolving field's steps 2-10 differ in
    # cost; a restored field's steps are all alike, three of them suffice)
    e2e = run.e2e(1 if args.mode == "persistent" else 0,
                  max(1, min(args.steps, EPISODE - 1)) if evolving else max(1, min(args.steps, 3)))

    mapped = None
    if args.map_tmax > 0 and not evolving:
        mapped = mapped_bench(h, F, args, run.T0, run.Y0, run.P, run.DT, run.T, run.Y, run.hio, run.ns, run.st,
                              flush, run.stream, meth, world, dev)
    secondary = None
    if args.workload == "lts" and not args.no_secondary and not args.cells and args.method == "rodas3":
        secondary = jet_key(h, dev, meth, oc, world, flush, clocks_path, local, rank)
    adj = None
    if not args.no_adjoint and not args.cells and args.method == "rodas3" and args.workload in ("lts", "jet", "large"):
        Fa, label = adjoint_fields(args.workload, m, F)
        adj = adjoint_bench(h, m, dev, Fa, label)
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return 0
    nsub, nac = res["nsub"], res["nacc"]
    launches_per_step = 4 if args.mode == "persistent" else 1
    line = {
        "metric": METRIC, "value": value, "unit": "reactor-steps/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * t_total / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": dict(config(args.workload, args.mode), n_cells=N,
                       warps_per_cell=int(h.info["auto_warps_per_cell"]), method=args.method,
                       cells_per_warp=args.cells_per_warp or int(h.info["auto_cells_per_warp"]),
                       tabulated_temperature_functions=(f"tables of relative tolerance {args.tabulate:g} (an "
                                                        "approximation)" if args.tabulate > 0 else "exact"),
                       kernels="mechanism-specialised (run-time compiled)" if args.specialized else "library"),
        "e2e": e2e,
        "gpu_launches": args.steps * launches_per_step,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                     "traffic": traffic,
                     "note": "FP64 pipe slots of the algorithm (opcount model, 2 flop per slot) / CUDA-event time of "
                             "the timed integrate steps; peak derived: 2 DFMA/clk/SM x 152 SM x 2.07 GHz; traffic: "
                             "DRAM bytes per launch scaled by cells from an ncu capture of the same workload's kernel "
                             "(null if the kernel sources changed since)"},
        "substeps": {"total_last_step": int(nsub.sum()), "mean_last_step": float(nsub.mean()),
                     "max_last_step": int(nsub.max()), "accepted_last_step": int(nac.sum()),
                     "timed_total": int(res["subs"]), "per_s": res["subs"] / t_total},
        "cell_status": {str(k): int(v) for k, v in zip(*np.unique(res["status"], return_counts=True))},
        "step_ms": res["step_ms"],
    }
    if res["episode_steps"] is not None:
        line["episode_step_of_timed_steps"] = res["episode_steps"]
    if args.tabulate > 0:
        line["tabulated"] = tabulation_deviation(run, args.tabulate)
    if res_other is not None:
        o = {"value": world * N * k_other / res_other["t"], "unit": "reactor-steps/s", "steps": k_other,
             "ms_per_step": 1e3 * res_other["t"] / k_other, "step_ms": res_other["step_ms"],
             "clocks": res_other["clocks"]}
        # the headline mode on exactly the same steps (its first k_other timed steps)
        t_same = sum(res["step_ms"][:k_other]) / 1e3
        o[f"{args.mode}_value_same_steps"] = world * N * k_other / t_same
        o[f"{args.mode}_over_{other}_same_steps"] = res_other["t"] / t_same
        line[other] = o
    if spec_info is not None:
        sp = dict(spec_info)
        if res_ab is not None:
            t_same = sum(res["step_ms"][:k_other]) / 1e3
            ab = "library" if args.specialized else "specialized"
            sp.update({f"{ab}_value": world * N * k_other / res_ab["t"], "unit": "reactor-steps/s",
                       "steps": k_other, f"{ab}_step_ms": res_ab["step_ms"],
                       "headline_value_same_steps": world * N * k_other / t_same,
                       # throughput ratio, specialised over library, on the same flow steps
                       "specialized_over_library": (t_same / res_ab["t"]) if not args.specialized
                       else (res_ab["t"] / t_same), "mode": args.mode})
        line["specialized"] = sp
    elif not one_warp:
        line["specialized"] = {"note": "not used: the specialised kernels run one cell per warp, this workload's "
                                       "choice differs"}
    if res["clocks"]:
        line["clocks"] = res["clocks"]
    if secondary is not None:
        line["jet"] = secondary
    if adj is not None:
        line["adjoint"] = adj
    if mapped is not None:
        line["mapped"] = mapped
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(m, F, args.workload, method=meth)
    print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


def tabulation_deviation(run, tol):
    """The tables' effect on one flow step from the initial field: largest relative difference of T and of
    every Y > 1e-12 between the tabulated and the exact integration (cells with the same substep count),
    and the share of cells whose step sequence changed."""
    import torch
    out = {}
    for key, kw in (("exact", {}), ("tab", run.tab)):
        run.reset()
        run.h.integrate(run.T, run.P, run.Y, run.DT, run.hio, run.ns, run.st, rtol=RTOL, atol=ATOL, mode=1,
                        method=run.meth, cells_per_warp=run.cpw, **kw)
        torch.cuda.synchronize()
        out[key] = (run.T.cpu().numpy(), run.Y.cpu().numpy().reshape(-1, run.N), run.ns.cpu().numpy())
    (Te, Ye, ne), (Tt, Yt, nt) = out["exact"], out["tab"]
    same = ne == nt
    big = np.abs(Ye) > 1e-12
    rel = np.where(big, np.abs(Yt - Ye) / np.where(big, np.abs(Ye), 1.0), 0.0)
    return {"tab_tol": tol, "max_rel_dT_same_steps": float(np.max(np.abs(Tt - Te)[same] / Te[same], initial=0.0)),
            "max_rel_dY_same_steps": float(rel[:, same].max(initial=0.0)),
            "cells_with_other_step_sequence": float(1.0 - same.mean()),
            "note": "one flow step from the initial field, persistent mode, tabulated vs exact"}


def jet_key(h, dev, meth, oc, world, flush, clocks_path, local, rank):
    """Secondary key: the 65,536-cell jet field (uniform dt = 1e-5 s, restored every step), persistent and
    plain, two timed steps each after one warm-up."""
    _, Fj = workload("jet", seed_offset=rank)
    rj = Runner(h, Fj, False, dev, meth, oc, world, flush, clocks_path, local)
    a = rj.run("persistent", 1, 2)
    b = rj.run("plain", 1, 2, count_work=False)
    Nj = Fj.n_cells
    from paper_2311_14941_gb300 import opcount
    achieved = opcount.FLOP_PER_SLOT * a["slots"] / a["t"] / 1e12
    return {"workload": WORKLOADS["jet"]["workload"], "n_cells": Nj, "steps": 2,
            "persistent": world * Nj * 2 / a["t"], "plain": world * Nj * 2 / b["t"], "unit": "reactor-steps/s",
            "persistent_over_plain": b["t"] / a["t"], "roofline_frac": achieved / opcount.fp64_peak_tflops(),
            "substeps_mean": float(a["nsub"].mean())}


if __name__ == "__main__":
    sys.exit(main())
