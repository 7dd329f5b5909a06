"""Zonal reference-cell mapping, written out plainly over the oracle's integrator -- TEST INFRASTRUCTURE.

Only the test-suite, the package smoke check and the benchmark's CPU legs use this module.

What it computes (Sec. 2.5: where the reactivity is low, the chemistry solution of a cell is mapped from
a reference cell instead of being integrated).  The paper names the technique without its rules; the
reading implemented here, and by the CUDA library's chem_integrate_mapped:
  - a cell is a candidate when its T is finite and below T_max;
  - a candidate's zone is the tuple (floor(T/dT), floor(Y_s/dY_s) for the listed species s, p, dt), the
    quotients in IEEE double arithmetic; a candidate with a non-finite key value or a quotient of
    magnitude 2^62 or more is not a candidate;
  - the cell of lowest index in each zone is its reference and is integrated; every other member takes
    the reference's change over dt added to its own state, the reference's status, no substeps of its
    own, and keeps its h;
  - every other cell is integrated as usual.
"""
from __future__ import annotations

import math

import numpy as np

_QMAX = 2.0 ** 62


def zone_key(T, p, dt, Ycol, T_max, dT, species, dY):
    """The zone of one cell (a hashable tuple), or None when the cell is not a candidate."""
    t = float(T)
    if not (math.isfinite(t) and t < T_max) or not (math.isfinite(float(p)) and math.isfinite(float(dt))):
        return None
    parts = []
    for x, d in [(t, dT)] + [(float(Ycol[s]), w) for s, w in zip(species, dY)]:
        if not math.isfinite(x):
            return None
        q = x / d
        if not abs(q) < _QMAX:
            return None
        parts.append(math.floor(q))
    return tuple(parts), float(p), float(dt)


def references(T, p, Y, dt, T_max, dT, species=(), dY=()):
    """ref[c]: the reference of cell c (c itself when c is integrated).  Y[k, c] species-major."""
    N = len(T)
    first = {}
    ref = np.arange(N)
    for c in range(N):
        key = zone_key(T[c], p[c], dt[c], Y[:, c], T_max, dT, species, dY)
        if key is None:
            continue
        if key in first:
            ref[c] = first[key]
        else:
            first[key] = c
    return ref


def integrate_mapped(oracle, T, p, Y, dt, mapping=None, rtol=1e-6, atol=1e-12, h_io=None, method=0, nthreads=0):
    """mapping: None or dict(T_max, dT, species, dY).  Returns dict T, Y, h, nsub, status, ref,
    n_integrated (arrays over all cells, Y[k, c])."""
    T = np.asarray(T, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    N = T.shape[0]
    h0 = np.zeros(N) if h_io is None else np.asarray(h_io, dtype=np.float64)
    if mapping is None:
        ref = np.arange(N)
    else:
        ref = references(T, p, Y, dt, mapping["T_max"], mapping["dT"], mapping.get("species", ()),
                         mapping.get("dY", ()))
    integ = np.flatnonzero(ref == np.arange(N))
    r = oracle.integrate_batch(T[integ], np.asarray(p)[integ], Y[:, integ], np.asarray(dt)[integ], rtol, atol,
                               h_io=h0[integ], method=method, nthreads=nthreads)
    T1, Y1, h1 = T.copy(), Y.copy(), h0.copy()
    nsub = np.zeros(N, dtype=np.int32)
    status = np.zeros(N, dtype=np.int32)
    T1[integ], Y1[:, integ], h1[integ] = r["T"], r["Y"], r["h"]
    nsub[integ], status[integ] = r["nsub"], r["status"]
    pos = np.full(N, -1)
    pos[integ] = np.arange(len(integ))
    for c in np.flatnonzero(ref != np.arange(N)):
        a = ref[c]
        j = pos[a]
        T1[c] = T[c] + (r["T"][j] - T[a])
        Y1[:, c] = Y[:, c] + (r["Y"][:, j] - Y[:, a])
        status[c] = r["status"][j]
    return dict(T=T1, Y=Y1, h=h1, nsub=nsub, status=status, ref=ref, n_integrated=int(len(integ)))
