"""Benchmark: reactor-steps/s of the stiff chemistry integrator on GB300.

One step = one chem_integrate call advancing every cell of the workload over its flow time step dt
(a "reactor-step" is one cell integrated over its dt).  Default workload: the 53-species / 325-reaction
synthetic mechanism on the 65,536-cell bimodal jet field (40 % unburnt, 60 % burnt, mixing layer),
uniform dt = 1e-5 s, FP64, rtol 1e-6 / atol 1e-12.  Every step starts from the same initial state
(restored by device copies inside the step).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--mode plain|persistent] [--impl reference]
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
NX, NY = 256, 256
DT = 1e-5
RTOL, ATOL = 1e-6, 1e-12


def workload(seed_offset=0):
    from paper_2311_14941_gb300 import synth
    m = synth.mechanism_methane_sized()
    F = synth.field_bimodal_jet(m, NX, NY, seed=2 + seed_offset, dt=DT)
    return m, F


def config(mode):
    return {"workload": "methane-sized 53sp/325rxn, 65536-cell bimodal jet field (40% unburnt 300-600 K, "
                        "60% burnt 1600-2200 K, tanh mixing layer), uniform dt=1e-5 s",
            "n_cells": NX * NY, "dt_s": DT, "rtol": RTOL, "atol": ATOL, "mode": mode,
            "l2": "flushed between timed steps (256 MiB write)", "state": "restored to the same initial field each step"}


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


def cpu_baseline(m, F, budget_s=12.0):
    """The oracle as it stands on this host's cores over a bounded sample of the workload's cells."""
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
        r = o.integrate_batch(S.T, S.p, S.Y, S.dt, RTOL, ATOL)
        t_used += time.perf_counter() - t0
        threads = r["threads"]
        done += len(sl)
        chunk = min(chunk * 2, 1024)
    return {"value": done / t_used, "unit": "reactor-steps/s", "cores": int(threads), "kind": "oracle",
            "sample": f"{done} seeded-random cells of the same 65536-cell field, integrated over dt=1e-5 s with "
                      f"OpenMP over cells ({t_used:.1f} s)"}


def adjoint_bench(h, m, dev, n_cells=4096):
    """Seconds per gradient: one chem_adjoint call (one cotangent vector, all cells, all 2R parameters) on
    igniting cells (T0 ~ U(1000, 1400) K, p ~ logU(1, 10) atm) integrated to t = 1e-3 s; objective = final
    T plus 5 seeded species mass fractions; checkpoints every 16 accepted steps."""
    import torch
    from paper_2311_14941_gb300 import synth
    F = synth.field_igniting(m, n_cells, seed=4, dt=1e-3)
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
    # warm-up on a few cells (module load, scratch growth happens on the full call below as well)
    h.adjoint(t(F.T[:64]), P[:64].contiguous(), t(F.Y[:, :64].reshape(-1)), D[:64].contiguous(), gT[:64].contiguous(),
              t(gYn[:, :64].reshape(-1)), gA, gE, st[:64].contiguous())
    torch.cuda.synchronize()
    T, Y = t(F.T), t(F.Y.reshape(-1))
    h.adjoint(T, P, Y, D, gT, gY, gA, gE, st)   # sizes the scratch for the full batch
    torch.cuda.synchronize()
    T, Y = t(F.T), t(F.Y.reshape(-1))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    h.adjoint(T, P, Y, D, gT, gY, gA, gE, st)
    e1.record()
    torch.cuda.synchronize()
    s = e0.elapsed_time(e1) / 1e3
    stat = st.cpu().numpy()
    return {"s_per_grad": s, "cells": N, "params": 2 * h.R, "cotangent": "final T (x1e-3) + 5 seeded species",
            "workload": "53sp/325rxn igniting cells, T0 1000-1400 K, p 1-10 atm, integrated to 1e-3 s, "
                        "checkpoints every 16 accepted steps",
            "cell_status": {str(k): int(v) for k, v in zip(*np.unique(stat, return_counts=True))},
            "grad_norm": float(torch.linalg.vector_norm(torch.cat([gA, gE])).item())}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    m, F = workload()
    from oracle.oracle import Oracle
    o = Oracle(m)
    rng = np.random.default_rng(13)
    per_step = 64
    for _ in range(args.warmup):
        S = F.subset(rng.choice(F.n_cells, per_step, replace=False))
        o.integrate_batch(S.T, S.p, S.Y, S.dt, RTOL, ATOL)
    t, threads = 0.0, 0
    for _ in range(args.steps):
        S = F.subset(rng.choice(F.n_cells, per_step, replace=False))
        t0 = time.perf_counter()
        r = o.integrate_batch(S.T, S.p, S.Y, S.dt, RTOL, ATOL)
        t += time.perf_counter() - t0
        threads = r["threads"]
    v = per_step * args.steps / t
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "reactor-steps/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": dict(config("oracle"), sample=f"{per_step} random cells per step"),
            "cpu_baseline": {"value": v, "unit": "reactor-steps/s", "cores": threads, "kind": "oracle",
                             "sample": f"{per_step} seeded-random cells of the workload per step"},
            "e2e": {"value": v, "unit": "reactor-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--mode", default="persistent", choices=["plain", "persistent"])
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cells", type=int, default=0, help="integrate only this many seeded-random cells (profiling)")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the adjoint seconds-per-gradient measurement")
    args = ap.parse_args()
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
    m, F = workload(seed_offset=rank)
    if args.cells:
        F = F.subset(np.sort(np.random.default_rng(5).permutation(F.n_cells)[: args.cells]))
    h = chem.create(m, local)
    oc = opcount.model(m, h.export_plan(0), h.export_plan(1))
    N = F.n_cells
    mode = 1 if args.mode == "persistent" else 0

    T0 = torch.tensor(F.T, device=dev)
    Y0 = torch.tensor(F.Y.reshape(-1), device=dev)
    P = torch.tensor(F.p, device=dev)
    DTs = torch.tensor(F.dt, device=dev)
    T = torch.empty_like(T0)
    Y = torch.empty_like(Y0)
    hio = torch.zeros(N, dtype=torch.float64, device=dev)
    ns = torch.zeros(N, dtype=torch.int32, device=dev)
    st = torch.zeros(N, dtype=torch.int32, device=dev)
    nacc = torch.zeros(N, dtype=torch.int32, device=dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)   # 256 MiB > L2
    stream = torch.cuda.current_stream()

    def step():
        # same initial state every step; nsub keeps the previous call's counts (the persistent mode's
        # sort key, as in consecutive flow steps)
        T.copy_(T0)
        Y.copy_(Y0)
        hio.zero_()
        h.integrate(T, P, Y, DTs, hio, ns, st, rtol=RTOL, atol=ATOL, mode=mode, naccept=nacc)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    torch.cuda.synchronize()
    with Clocks(os.path.join(ROOT, "gpurun_out" if os.path.isdir(os.path.join(ROOT, "gpurun_out")) else ".",
                             f"bench_clocks_r{rank}.csv")) as ck:
        for i in range(args.steps):
            flush.fill_(float(i))
            evs[i][0].record(stream)
            step()
            evs[i][1].record(stream)
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    step_ms = [a.elapsed_time(b) for a, b in evs]
    t_total = sum(step_ms) / 1e3
    t_max = torch.tensor([t_total], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(t_max, op=dist.ReduceOp.MAX)
    t_total = float(t_max.item())
    value = world * N * args.steps / t_total
    status = st.cpu().numpy()
    nsub = ns.cpu().numpy()
    nac = nacc.cpu().numpy()

    # roofline: algorithmic FP64 work of one launch / its duration
    slots = float(oc.cell_slots(nsub, nac).sum())
    launch_s = t_total / args.steps
    achieved = opcount.FLOP_PER_SLOT * slots / launch_s / 1e12
    peak = opcount.fp64_peak_tflops()

    # end to end through the ABI with host buffers (pinned), copies inside the timed region
    Th = torch.tensor(F.T).pin_memory()
    Yh = torch.tensor(F.Y.reshape(-1)).pin_memory()
    Ph = torch.tensor(F.p).pin_memory()
    Dh = torch.tensor(F.dt).pin_memory()
    To = torch.empty_like(Th).pin_memory()
    Yo = torch.empty_like(Yh).pin_memory()
    So = torch.empty(N, dtype=torch.int32).pin_memory()
    e2e_steps = max(1, min(args.steps, 3))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        T.copy_(Th, non_blocking=True)
        Y.copy_(Yh, non_blocking=True)
        P.copy_(Ph, non_blocking=True)
        DTs.copy_(Dh, non_blocking=True)
        hio.zero_()
        h.integrate(T, P, Y, DTs, hio, ns, st, rtol=RTOL, atol=ATOL, mode=mode)
        To.copy_(T, non_blocking=True)
        Yo.copy_(Y, non_blocking=True)
        So.copy_(st, non_blocking=True)
        torch.cuda.synchronize()
    t_e2e = time.perf_counter() - t0
    h2d = (Th.numel() + Yh.numel() + Ph.numel() + Dh.numel()) * 8
    d2h = (To.numel() + Yo.numel()) * 8 + So.numel() * 4

    if rank != 0:
        return 0
    line = {
        "metric": METRIC, "value": value, "unit": "reactor-steps/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * t_total / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": dict(config(args.mode), n_cells=N),
        "e2e": {"value": world * N * e2e_steps / t_e2e, "unit": "reactor-steps/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": args.steps,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                     "traffic": None,
                     "note": "FP64 pipe slots of the algorithm (opcount model, 2 flop per slot) / CUDA-event time of "
                             "the integrate launch; peak derived: 2 DFMA/clk/SM x 152 SM x 2.07 GHz"},
        "substeps": {"total": int(nsub.sum()), "mean": float(nsub.mean()), "max": int(nsub.max()),
                     "accepted": int(nac.sum())},
        "cell_status": {str(k): int(v) for k, v in zip(*np.unique(status, return_counts=True))},
        "step_ms": step_ms,
    }
    ck_s = ck.summary(local)
    if ck_s:
        line["clocks"] = ck_s
    if not args.no_adjoint and not args.cells:
        line["adjoint"] = adjoint_bench(h, m, dev)
    if not args.no_cpu_baseline and world >= 1:
        line["cpu_baseline"] = cpu_baseline(m, F)
    print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
