"""Algorithmic FP64 work of the integrator, for the roofline.

The path is bound by the FP64 pipe (2 DFMA lanes per clock per SM on GB300), not by memory or tensor
cores.  Work is counted in FP64 pipe slots of an ideal implementation of the same algorithm: every
useful add, multiply or fused multiply-add is one slot; a divide, exp or log is charged the slots it
occupies on this GPU, measured relative to DFMA by a microbenchmark (divide 6, sqrt 6, pow 60; exp 11
and log 13 for the library's table-driven functions, against 18 and 34 for the CUDA math library's).  Idle lanes, redundant recomputation and index arithmetic are not counted.  Reported
as TFLOP/s-equivalent = 2 x slots/s, so a kernel that kept the pipe busy with useful DFMAs would read
the FP64 peak: 2 slots/clk/SM x 152 SMs x 2.07 GHz x 2 = 1.259 TFLOP/s.

Counts are per cell and per unit of work:
  attempt : one RODAS3 attempt given J (LU build + factor, z = A^-1 u, 4 stage solves with the
            Sherman-Morrison correction, 2 right-hand sides, stage vectors, error norm, control)
  jac     : one Jacobian evaluation (right-hand side at y included: it is f0)
A cell that made `nsub` attempts of which `nacc` were accepted evaluated J `nacc` times when it ended
with an accepted step (J is refreshed only after an acceptance), so
  slots(cell) = nsub * attempt + nacc * jac.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

DIV, EXP, LOG, SQRT, POW = 6, 11, 13, 6, 60
SLOTS_PER_CLK_SM = 2
FLOP_PER_SLOT = 2


def fp64_peak_tflops(n_sm: int = 152, clk_ghz: float = 2.07) -> float:
    return SLOTS_PER_CLK_SM * n_sm * clk_ghz * FLOP_PER_SLOT / 1e3


@dataclass
class OpCount:
    f_eval: float
    jac: float
    attempt: float
    lu: float
    solve: float

    def cell_slots(self, nsub, nacc):
        return np.asarray(nsub, dtype=np.float64) * self.attempt + np.asarray(nacc, dtype=np.float64) * self.jac


def model(desc, lu_prog: np.ndarray, sv_prog: np.ndarray, method: int = 0) -> OpCount:
    """desc: flat mechanism (synth.MechDesc); lu_prog/sv_prog: the exported warp programs; method 0 RODAS3
    (2 new right-hand sides, z and 4 stage solves per attempt), 1 ROS2 (1 right-hand side, z and 2 stage
    solves), 2 RODAS4 (5 right-hand sides, z and 6 stage solves)."""
    n = len(desc.W)
    R = len(desc.A)
    m = n + 1
    rt = np.asarray(desc.rtype)
    # ---- right-hand side
    species = n * (4 + 5 + 7 + EXP + DIV + 1 + 1 + 1 + 1)       # cp, h, g polys, exp, 1/exp, Y/W, sums, C
    cell = LOG + 3 * DIV + 8
    rx = 0.0
    omega_terms = 0
    jac_rx = 0.0
    dtil_terms = 0
    n_dslot = 0
    cols_per_rx = []
    for r in range(R):
        ro = int(np.sum(desc.reac_nu[desc.reac_ptr[r]:desc.reac_ptr[r + 1]]))
        po = int(np.sum(desc.prod_nu[desc.prod_ptr[r]:desc.prod_ptr[r + 1]]))
        neff = int(desc.eff_ptr[r + 1] - desc.eff_ptr[r]) if rt[r] != 0 else 0
        c = 2 + EXP + (ro - 1) + (po - 1) + neff + 2
        if desc.reversible[r]:
            c += (ro + po - 1) + abs(po - ro) + 1
        if rt[r] == 1:
            c += 1
        if rt[r] == 2:
            T2 = desc.troe[r][3] > 0
            c += 2 + LOG + 2 + EXP + (2 + 2 * EXP) + ((EXP + 1) if T2 else 0) + 2 + (LOG + 1) + 2 + 2 + DIV + 1 + \
                (1 + DIV) + 1 + (EXP + 1) + (1 + DIV) + 3
        rx += c
        nu = {}
        for i in range(desc.reac_ptr[r], desc.reac_ptr[r + 1]):
            nu[int(desc.reac_sp[i])] = nu.get(int(desc.reac_sp[i]), 0) - int(desc.reac_nu[i])
        for i in range(desc.prod_ptr[r], desc.prod_ptr[r + 1]):
            nu[int(desc.prod_sp[i])] = nu.get(int(desc.prod_sp[i]), 0) + int(desc.prod_nu[i])
        nz = sum(1 for v in nu.values() if v != 0)
        omega_terms += nz
        cols = set(desc.reac_sp[desc.reac_ptr[r]:desc.reac_ptr[r + 1]].tolist()) | \
            set(desc.prod_sp[desc.prod_ptr[r]:desc.prod_ptr[r + 1]].tolist())
        if rt[r] != 0:
            cols |= set(desc.eff_sp[desc.eff_ptr[r]:desc.eff_ptr[r + 1]].tolist())
        ncol = len(cols)
        n_dslot += ncol
        dtil_terms += nz * ncol
        # Jacobian extras of the reaction: rate derivatives, dq/dT, derivative slots
        jr = 2 + 4 + 2 + 5 + (3 if ro == 3 else 0) + (3 if po == 3 else 0) + ncol * 3
        if desc.reversible[r]:
            jr += (ro + po - 1) + 2
        if rt[r] == 2:
            jr += 30 + DIV + 2
        jac_rx += jr
    f_eval = species + cell + rx + omega_terms + n * 3 + 6 + DIV
    # ---- Jacobian (includes f at y)
    nY = len({(k, j) for k, j in _entries(desc)})
    jac = f_eval + jac_rx + omega_terms + dtil_terms + 2 * nY + nY + n * 16 + n * 4 + 20 + 3 * DIV
    # ---- linear algebra from the compiled programs (useful lane-ops only)
    lp = lu_prog.reshape(-1, 32, 4)
    live = lp[:, :, 1] != 65535
    kinds = lp[:, 0, 0]
    n_upd = int(live[kinds == 2].sum())
    n_scl = int(live[kinds == 1].sum())
    n_rcp = int(live[kinds == 0].sum())
    lu = n_upd + n_scl + n_rcp * DIV + m
    sp = sv_prog.reshape(-1, 32, 4)
    solve = float((sp[:, :, 1] != 65535).sum())
    sm = solve + 2 * m
    if method == 1:
        attempt = lu + (solve + m + DIV) + 2 * sm + f_eval + m * (1 + 1 + 2 + 2) + m * (2 + DIV + 1) + SQRT + POW + 10
    elif method == 2:
        # stage points and coefficient sums: 2 + 5 + 7 + 9 + 8 per component, then solution and error
        attempt = (lu + (solve + m + DIV) + 6 * sm + 5 * f_eval + m * (2 + 5 + 7 + 9 + 8) + m * (2 + DIV + 1) +
                   SQRT + POW + 10)
    else:
        attempt = (lu + (solve + m + DIV) + 4 * sm + 2 * f_eval + m * (1 + 1 + 3 + 2 + 4 + 3) + m * (1 + DIV + 1) +
                   SQRT + POW + 10)
    return OpCount(float(f_eval), float(jac), float(attempt), float(lu), float(solve))


def _entries(desc):
    n = len(desc.W)
    rt = np.asarray(desc.rtype)
    out = {(k, k) for k in range(n)}
    for r in range(len(desc.A)):
        nu = {}
        for i in range(desc.reac_ptr[r], desc.reac_ptr[r + 1]):
            nu[int(desc.reac_sp[i])] = nu.get(int(desc.reac_sp[i]), 0) - int(desc.reac_nu[i])
        for i in range(desc.prod_ptr[r], desc.prod_ptr[r + 1]):
            nu[int(desc.prod_sp[i])] = nu.get(int(desc.prod_sp[i]), 0) + int(desc.prod_nu[i])
        cols = set(desc.reac_sp[desc.reac_ptr[r]:desc.reac_ptr[r + 1]].tolist()) | \
            set(desc.prod_sp[desc.prod_ptr[r]:desc.prod_ptr[r + 1]].tolist())
        if rt[r] != 0:
            cols |= set(desc.eff_sp[desc.eff_ptr[r]:desc.eff_ptr[r + 1]].tolist())
        for k, v in nu.items():
            if v != 0:
                for j in cols:
                    out.add((k, j))
    return out
