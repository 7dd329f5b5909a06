"""Host-side logic of the CUDA library, checked without a GPU: the exported C ABI, the compiled
sparse pattern, and the warp elimination / substitution programs executed step by step in numpy."""
import ctypes

import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2311_14941_gb300 import chem, synth
from tests import tinymech as tm

MECHS = {"small": synth.mechanism_small, "mid": synth.mechanism_methane_sized, "large": synth.mechanism_large}


@pytest.fixture(scope="module", params=list(MECHS))
def compiled(request):
    m = MECHS[request.param]()
    return m, chem.create(m, device=-1)


def test_library_exports_every_declared_symbol():
    L = ctypes.CDLL(chem._build.build())
    names = chem.declared_functions()
    assert len(names) >= 9
    for name in names:
        assert hasattr(L, name), name


def _internal_S_dense(h, S_csr):
    """Map CSR-ordered S values to the internal order and to a dense matrix."""
    rp, ci = h.jacobian_pattern()
    m = h.m
    dense = np.zeros((m, m))
    for r in range(m):
        dense[r, ci[rp[r]:rp[r + 1]]] = S_csr[rp[r]:rp[r + 1]]
    s_out = h.export_plan(5)
    return S_csr[s_out], dense


def _run_elimination(prog, LU, dinv, width=32):
    P = prog.reshape(-1, width, 4)
    for st in P:
        kind = st[0, 0]
        assert np.all(st[:, 0] == kind), "every lane's op carries the step's kind"
        live = st[st[:, 1] != 65535]
        t, a, b = live[:, 1], live[:, 2], live[:, 3]
        assert len(np.unique(t)) == len(t), "two lanes write one target in a step"
        # lanes of one step run unordered (two warps per cell are not in lockstep): no lane of an update
        # step may read a factor entry that another lane of the step writes (scale and reciprocal steps
        # read only their own target and the 1/pivot array)
        if kind == 2:
            assert not np.isin(t, np.concatenate([a, b])).any(), "a step reads an entry it writes"
        if kind == 2:
            LU[t] = LU[t] - LU[a] * LU[b]
        elif kind == 1:
            LU[t] = LU[t] * dinv[a]
        else:
            dinv[t] = 1.0 / LU[a]


def _run_solve(prog, LU, dinv, x, width=32):
    P = prog.reshape(-1, width, 4)
    for st in P:
        kind = st[0, 0]
        assert np.all(st[:, 0] == kind)
        live = st[st[:, 1] != 65535]
        t, a, b = live[:, 1], live[:, 2], live[:, 3]
        assert len(np.unique(t)) == len(t)
        if kind == 2:
            assert not np.isin(t, b).any(), "a step reads a vector entry it writes"
        if kind == 2:
            x[t] = x[t] - LU[a] * x[b]
        else:
            x[t] = x[t] * dinv[a]


PLANS = {32: (0, 1, 6), 64: (8, 9, 10), 16: (11, 12, 13)}   # width -> elimination, solve, transposed solve


@pytest.mark.parametrize("width", [32, 64, 16])
def test_programs_reproduce_dense_solve(compiled, width):
    """I/(h gamma) - S factored and solved by the warp programs (one warp, two warps or half a warp per
    cell) equals numpy's dense solve."""
    m_, h = compiled
    plan_lu, plan_sv, _ = PLANS[width]
    rng = np.random.default_rng(1)
    info = h.info
    S_csr = rng.standard_normal(info["nnz_S"])
    S_int, S_dense = _internal_S_dense(h, S_csr)
    gh = 3.0 * np.abs(S_dense).sum(axis=1).max()
    A = gh * np.eye(h.m) - S_dense
    lu_src = h.export_plan(4)
    LU = np.where(lu_src >= 0, -S_int[np.maximum(lu_src, 0)], 0.0)
    perm = h.export_plan(2)
    pat = h.export_plan(3)
    rowptr, col = pat[: h.m + 1], pat[h.m + 1:]
    for p in range(h.m):
        for sl in range(rowptr[p], rowptr[p + 1]):
            if col[sl] == p:
                LU[sl] += gh
    dinv = np.zeros(h.m)
    _run_elimination(h.export_plan(plan_lu), LU, dinv, width)
    assert sorted(perm.tolist()) == list(range(h.m)) and perm[-1] == 0      # T eliminated last
    for _ in range(3):
        bvec = rng.standard_normal(h.m)
        x = bvec.copy()
        _run_solve(h.export_plan(plan_sv), LU, dinv, x, width)
        ref = np.linalg.solve(A, bvec)
        assert np.max(np.abs(x - ref)) <= 1e-12 * np.max(np.abs(ref))


@pytest.mark.parametrize("width", [32, 64, 16])
def test_transposed_program_solves_the_transpose(compiled, width):
    """The transposed substitution program applied to the same factor solves A^T x = b."""
    m_, h = compiled
    plan_lu, _, plan_t = PLANS[width]
    rng = np.random.default_rng(2)
    S_csr = rng.standard_normal(h.info["nnz_S"])
    S_int, S_dense = _internal_S_dense(h, S_csr)
    gh = 3.0 * np.abs(S_dense).sum(axis=1).max()
    A = gh * np.eye(h.m) - S_dense
    lu_src = h.export_plan(4)
    LU = np.where(lu_src >= 0, -S_int[np.maximum(lu_src, 0)], 0.0)
    pat = h.export_plan(3)
    rowptr, col = pat[: h.m + 1], pat[h.m + 1:]
    for p in range(h.m):
        for sl in range(rowptr[p], rowptr[p + 1]):
            if col[sl] == p:
                LU[sl] += gh
    dinv = np.zeros(h.m)
    _run_elimination(h.export_plan(plan_lu), LU, dinv, width)
    for _ in range(3):
        bvec = rng.standard_normal(h.m)
        x = bvec.copy()
        _run_solve(h.export_plan(plan_t), LU, dinv, x, width)
        ref = np.linalg.solve(A.T, bvec)
        assert np.max(np.abs(x - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_pattern_holds_the_sparse_part_of_the_exact_jacobian(compiled):
    """Outside the compiled pattern the oracle's exact Jacobian must be the rank-one density coupling
    u_i Wbar / W_j (the same u_i for every column of a row)."""
    m, h = compiled
    o = Oracle(m)
    rp, ci = h.jacobian_pattern()
    inside = np.zeros((h.m, h.m), bool)
    for r in range(h.m):
        inside[r, ci[rp[r]:rp[r + 1]]] = True
    assert inside[0].all() and inside[:, 0].all() and np.diag(inside).all()
    F = synth.field_uniform_random(m, 3, seed=2)
    for c in range(3):
        J, G = o.jacobian(F.T[c], F.p[c], F.Y[:, c], want_gross=True)
        Wbar = 1.0 / np.sum(F.Y[:, c] / m.W)
        v = np.r_[0.0, Wbar / m.W]
        for i in range(1, h.m):
            out = np.where(~inside[i])[0]
            if len(out) == 0:
                continue
            u = J[i, out] / v[out]
            scale = np.max(np.abs(G[i])) + 1e-300
            assert np.max(np.abs(u - np.median(u)) * v[out]) <= 1e-12 * scale


def _bad(mod):
    m = synth.mechanism_small()
    mod(m)
    return m


@pytest.mark.parametrize("name,mod", [
    ("unbalanced", lambda m: m.prod_sp.__setitem__(0, (m.prod_sp[0] + 1) % m.n_species)),
    ("negative W", lambda m: m.W.__setitem__(2, -0.01)),
    ("nan A", lambda m: m.A.__setitem__(3, np.nan)),
    ("species out of range", lambda m: m.reac_sp.__setitem__(1, 99)),
    ("zero coefficient", lambda m: m.reac_nu.__setitem__(0, 0)),
    ("bad Troe T3", lambda m: m.troe.__setitem__((0, 1), -5.0)),
])
def test_invalid_descriptions_are_rejected(name, mod):
    with pytest.raises(chem.ChemError) as ei:
        chem.create(_bad(mod), device=-1)
    assert "status 1" in str(ei.value)


def test_compute_on_host_only_handle_fails_loudly():
    import torch
    h = chem.create(synth.mechanism_small(), device=-1)
    with pytest.raises((chem.ChemError, ValueError)):
        t = torch.zeros(4, dtype=torch.float64)
        h.rates(t, t, t, t, t)
