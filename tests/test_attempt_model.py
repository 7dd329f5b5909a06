"""A CPU model of one device attempt against the oracle's step, for RODAS3, ROS2 and RODAS4.

The model runs what the kernels run, in numpy:
  - the exported elimination and substitution programs, step by step, on A = I/(h gamma) - S;
  - the Sherman-Morrison correction for the rank-one part u v^T of J;
  - the transformed stages with the constants parsed from device.cuh.
The oracle instead takes a dense LU of I - h gamma J and the k-form.  Agreement to rounding checks
the structure of the device algorithm on the CPU (stage order, coefficient use, the split of J, the
programs' dependences).  It is a check of the design, not of the compiled kernels, which the GPU
parity tests compare with the oracle."""
import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2311_14941_gb300 import chem, synth
from tests.test_device_constants import _constants
from tests.test_host_plan import _run_elimination, _run_solve


def _split(h, m, o, T, p, Y):
    """J = S + u v^T with S in the compiled pattern (v_0 = 0, v_j = Wbar / W_j; u_i from the entries
    outside the pattern, 0 for rows that lie wholly inside it)."""
    J = o.jacobian(T, p, Y)
    mm = h.m
    rp, ci = h.jacobian_pattern()
    inside = np.zeros((mm, mm), bool)
    for r in range(mm):
        inside[r, ci[rp[r]:rp[r + 1]]] = True
    Wbar = 1.0 / np.sum(Y / m.W)
    v = np.r_[0.0, Wbar / m.W]
    u = np.zeros(mm)
    for i in range(mm):
        out = np.where(~inside[i])[0]
        if len(out):
            u[i] = np.median(J[i, out] / v[out])
    S = np.where(inside, J - np.outer(u, v), 0.0)
    return S, u, v, rp, ci


def _factor(h, S, rp, ci, gh):
    """The device's factor of A = gh I - S by the exported elimination program (one warp per cell)."""
    S_csr = np.concatenate([S[r, ci[rp[r]:rp[r + 1]]] for r in range(h.m)])
    S_int = S_csr[h.export_plan(5)]
    lu_src = h.export_plan(4)
    LU = np.where(lu_src >= 0, -S_int[np.maximum(lu_src, 0)], 0.0)
    pat = h.export_plan(3)
    rowptr, col = pat[: h.m + 1], pat[h.m + 1:]
    for q in range(h.m):
        for sl in range(rowptr[q], rowptr[q + 1]):
            if col[sl] == q:
                LU[sl] += gh
    dinv = np.zeros(h.m)
    _run_elimination(h.export_plan(0), LU, dinv)
    sv = h.export_plan(1)

    def solve(b):
        x = np.array(b, dtype=np.float64)
        _run_solve(sv, LU, dinv, x)
        return x
    return solve


def _attempt(method, K, f, y, hstep, solve_for, u, v):
    g = {0: K["RG"], 1: K["RG2"], 2: K["RG4"]}[method]
    solve = solve_for(1.0 / (hstep * g))
    z = solve(u)
    iden = 1.0 / (1.0 - v @ z)

    def sm(b):
        x = solve(b)
        return x + z * ((v @ x) * iden)
    ih = 1.0 / hstep
    f0 = f(y)
    U1 = sm(f0)
    if method == 0:
        U2 = sm(f0 + K["C21"] * ih * U1)
        U3 = sm(f(y + K["A31"] * U1) + ih * (K["C31"] * U1 + K["C32"] * U2))
        U4 = sm(f(y + K["A41"] * U1 + K["A43"] * U3) + ih * (K["C41"] * U1 + K["C42"] * U2 + K["C43"] * U3))
        return y + K["M1"] * U1 + K["M3"] * U3 + K["M4"] * U4, U4
    if method == 1:
        U2 = sm(f(y + K["R2_A21"] * U1) + K["R2_C21"] * ih * U1)
        return y + K["R2_M1"] * U1 + K["R2_M2"] * U2, K["R2_E"] * (U1 + U2)
    a = lambda i, j: K[f"R4_A{i}{j}"]
    c = lambda i, j: K[f"R4_C{i}{j}"]
    U = [U1]
    yt = y
    for i in range(2, 6):
        yt = y + sum(a(i, j) * U[j - 1] for j in range(1, i))
        U.append(sm(f(yt) + ih * sum(c(i, j) * U[j - 1] for j in range(1, i))))
    y6 = yt + U[4]
    U6 = sm(f(y6) + ih * sum(c(6, j) * U[j - 1] for j in range(1, 6)))
    return y6 + U6, U6


@pytest.mark.parametrize("mech,hstep", [("small", 1e-11), ("mid", 1e-10)])
@pytest.mark.parametrize("method", [0, 1, 2])
def test_device_attempt_model_matches_the_oracle_step(mech, hstep, method):
    m = synth.mechanism_small() if mech == "small" else synth.mechanism_methane_sized()
    h = chem.create(m, device=-1)
    o = Oracle(m)
    K = _constants()
    F = synth.field_uniform_random(m, 3, seed=7) if mech == "small" else \
        synth.field_bimodal_jet(m, 8, 8, seed=2).subset([0, 20, 40])
    for c in range(F.n_cells):
        T, p, Y = F.T[c], F.p[c], F.Y[:, c]
        S, u, v, rp, ci = _split(h, m, o, T, p, Y)
        assert np.allclose(S + np.outer(u, v), o.jacobian(T, p, Y), rtol=1e-12,
                           atol=1e-12 * np.abs(o.jacobian(T, p, Y)).max())
        y = o.state(T, Y)
        f = lambda yy: o.rhs(yy[0], p, yy[1:])["f"]
        yn, err = _attempt(method, K, f, y, hstep, lambda gh: _factor(h, S, rp, ci, gh), u, v)
        yo, eo = o.step(y, p, hstep, method=method)
        assert np.all(np.isfinite(yo))
        # T to 1e-12 relative; Y to 1e-10 relative or a few ulps of the cell's largest mass fraction (the
        # two sides round differently, and the differences measured are at most 6e-17 in Y)
        assert abs(yn[0] - yo[0]) <= 1e-12 * abs(yo[0])
        tol = 1e-10 * np.abs(yo[1:]) + 1e-15 * np.max(np.abs(y[1:]))
        assert np.all(np.abs(yn[1:] - yo[1:]) <= tol)
        assert np.max(np.abs(err - eo)) <= 1e-8 * np.max(np.abs(eo)) + 1e-15 * np.max(np.abs(y))
