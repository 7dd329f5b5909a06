"""Discrete adjoint (chem_adjoint) against the oracle's complex-step derivatives of its own replayed
integration (frozen accepted step sizes), and against central differences of the GPU forward map.

The objective of one call is L = sum_c (gT_c T_c(dt) + sum_k gY_kc Y_kc(dt)).  Per cell, dL/d(ln A_j),
dL/d(Ea_j) and dL/d(initial state) of the discrete map are compared with the oracle's complex step
(exact to roundoff).  The two step sequences agree to rounding (the forward parity tests check that),
so the derivatives agree to a tolerance set by that rounding, 1e-7 relative to the gradient's norm.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle.oracle import Oracle  # noqa: E402
from paper_2311_14941_gb300 import chem, synth  # noqa: E402


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def _adjoint(h, F, gT, gY, dev, **kw):
    N = F.n_cells
    t = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)
    T, Y = t(F.T), t(F.Y.reshape(-1))
    gA = torch.zeros(h.R, dtype=torch.float64, device=dev)
    gE = torch.zeros(h.R, dtype=torch.float64, device=dev)
    gc = torch.zeros(2 * h.R * N, dtype=torch.float64, device=dev)
    gT0 = torch.zeros(N, dtype=torch.float64, device=dev)
    gY0 = torch.zeros(h.n * N, dtype=torch.float64, device=dev)
    st = torch.zeros(N, dtype=torch.int32, device=dev)
    h.adjoint(T, t(F.p), Y, t(F.dt), t(gT), t(gY.reshape(-1)), gA, gE, st, grad_cell=gc, gT0=gT0, gY0=gY0, **kw)
    torch.cuda.synchronize()
    return dict(T=T.cpu().numpy(), Y=Y.cpu().numpy().reshape(h.n, N), gA=gA.cpu().numpy(), gE=gE.cpu().numpy(),
                gc=gc.cpu().numpy().reshape(2 * h.R, N), gT0=gT0.cpu().numpy(), gY0=gY0.cpu().numpy().reshape(h.n, N),
                status=st.cpu().numpy())


def _oracle_grads(o, F, c, gT, gY, params):
    """Complex-step dL/dtheta for the listed (kind, j) and dL/dy0 through the oracle's replayed steps."""
    out = o.integrate(F.T[c], F.p[c], F.Y[:, c], F.dt[c], trace=True)
    hs = out["trace_h"][out["trace_acc"] == 1]
    y0 = o.state(F.T[c], F.Y[:, c])
    wvec = np.r_[gT[c], gY[:, c]]
    res = {}
    for kind, j in params:
        res[(kind, j)] = wvec @ o.replay_sens_cs(y0, F.p[c], hs, kind, j)
    return res, out


def _check_cell(o, F, c, g, gT, gY, params, tol=1e-7):
    ref, out = _oracle_grads(o, F, c, gT, gY, params)
    R = o.R
    got = {}
    for kind, j in params:
        got[(kind, j)] = g["gc"][j, c] if kind == 0 else g["gc"][R + j, c] if kind == 1 else \
            (g["gT0"][c] if j == 0 else g["gY0"][j - 1, c])
    for kind in (0, 1, 2):
        keys = [k for k in params if k[0] == kind]
        if not keys:
            continue
        r = np.array([ref[k] for k in keys])
        v = np.array([got[k] for k in keys])
        scale = np.max(np.abs(r)) + 1e-300
        assert np.max(np.abs(v - r)) <= tol * scale, (kind, c, np.max(np.abs(v - r)) / scale)
    # the adjoint's forward pass returns the same final state as chem_integrate / the oracle
    assert abs(g["T"][c] - out["T"]) <= 1e-8 * out["T"]


def test_adjoint_small_mechanism_all_parameters(dev):
    m = synth.mechanism_small()
    h, o = chem.create(m, 0), Oracle(m)
    F = synth.field_uniform_random(m, 6, seed=31, dt=2e-7)
    rng = np.random.default_rng(0)
    gT = rng.standard_normal(F.n_cells) * 1e-3
    gY = rng.standard_normal((m.n_species, F.n_cells))
    g = _adjoint(h, F, gT, gY, dev)
    assert np.all(g["status"] == 0)
    params = [(0, j) for j in range(m.n_reactions)] + [(1, j) for j in range(m.n_reactions)] + \
             [(2, i) for i in range(m.n_species + 1)]
    for c in range(3):
        _check_cell(o, F, c, g, gT, gY, params)
    # summed over cells
    assert np.allclose(g["gA"], g["gc"][: m.n_reactions].sum(axis=1), rtol=1e-12, atol=0)


def test_adjoint_methane_sized_igniting_subset(dev):
    """Igniting cells (1000-1400 K, 1-10 atm), objective = T and 5 seeded species (checkpoints every 16)."""
    m = synth.mechanism_methane_sized()
    h, o = chem.create(m, 0), Oracle(m)
    F = synth.field_igniting(m, 8, seed=4, dt=2e-6)
    sel = synth.cotangent_species(m, 5, seed=4)
    gT = np.full(F.n_cells, 1e-3)
    gY = np.zeros((m.n_species, F.n_cells))
    gY[sel] = 1.0
    g = _adjoint(h, F, gT, gY, dev, ckpt_every=16)
    assert np.all(g["status"] == 0)
    rng = np.random.default_rng(1)
    for c in (0, 5):
        r = o.rhs(F.T[c], F.p[c], F.Y[:, c])
        active = list(np.argsort(-(np.abs(r["qf"]) + np.abs(r["qr"])))[:6])
        js = sorted(set(int(j) for j in active) | set(int(j) for j in rng.choice(m.n_reactions, 6, replace=False)))
        params = [(0, j) for j in js] + [(1, j) for j in js] + [(2, i) for i in (0, 1, 5, 20)]
        _check_cell(o, F, c, g, gT, gY, params)


def test_adjoint_matches_central_differences_of_gpu_forward(dev):
    """dL/dlnA_j summed over cells vs central differences of chem_integrate with shifted parameters
    (adaptive steps free to move: agreement to the integration tolerance, not to roundoff)."""
    m = synth.mechanism_small()
    h = chem.create(m, 0)
    F = synth.field_uniform_random(m, 64, seed=5, dt=1e-6)
    gT = np.full(F.n_cells, 1e-3)
    gY = np.zeros((m.n_species, F.n_cells))
    gY[[1, 4]] = 1.0
    g = _adjoint(h, F, gT, gY, dev, rtol=1e-9, atol=1e-15, tape_steps=30000)
    assert np.all(g["status"] == 0)
    t = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)

    def L(dl):
        T, Y = t(F.T), t(F.Y.reshape(-1))
        N = F.n_cells
        h.set_params(dlnA=t(dl))
        h.integrate(T, t(F.p), Y, t(F.dt), torch.zeros(N, dtype=torch.float64, device=dev),
                    torch.zeros(N, dtype=torch.int32, device=dev), torch.zeros(N, dtype=torch.int32, device=dev),
                    rtol=1e-9, atol=1e-15)
        h.set_params()
        torch.cuda.synchronize()
        Tn, Yn = T.cpu().numpy(), Y.cpu().numpy().reshape(m.n_species, N)
        return float(gT @ Tn + np.sum(gY * Yn))

    for j in np.argsort(-np.abs(g["gA"]))[:4]:
        e = np.zeros(m.n_reactions)
        e[j] = 1e-5
        fd = (L(e) - L(-e)) / 2e-5
        assert abs(fd - g["gA"][j]) <= 1e-4 * abs(g["gA"][j]), (j, fd, g["gA"][j])


def test_autograd_function_routes_to_the_adjoint(dev):
    """torch.autograd through ChemIntegrate gives the adjoint's gradients for ln A / Ea shifts and the
    initial state; with zero shifts the forward equals chem_integrate."""
    from paper_2311_14941_gb300 import autograd as ag
    m = synth.mechanism_small()
    h = chem.create(m, 0)
    F = synth.field_uniform_random(m, 16, seed=8, dt=3e-7)
    t = lambda a, g=False: torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev, requires_grad=g)
    T0, Y0 = t(F.T, True), t(F.Y, True)
    dlnA = torch.zeros(m.n_reactions, dtype=torch.float64, device=dev, requires_grad=True)
    dEa = torch.zeros(m.n_reactions, dtype=torch.float64, device=dev, requires_grad=True)
    T, Y, st = ag.integrate(h, T0, t(F.p), Y0, t(F.dt), dlnA, dEa)
    loss = 1e-3 * T.sum() + Y[2].sum() - 0.5 * Y[5].sum()
    loss.backward()
    gT = np.full(F.n_cells, 1e-3)
    gY = np.zeros((m.n_species, F.n_cells))
    gY[2] = 1.0
    gY[5] = -0.5
    ref = _adjoint(h, F, gT, gY, dev)
    assert np.array_equal(T.detach().cpu().numpy(), ref["T"])
    assert np.allclose(dlnA.grad.cpu().numpy(), ref["gA"], rtol=1e-13, atol=0)
    assert np.allclose(dEa.grad.cpu().numpy(), ref["gE"], rtol=1e-13, atol=0)
    assert np.allclose(T0.grad.cpu().numpy(), ref["gT0"], rtol=1e-13, atol=0)
    assert np.allclose(Y0.grad.cpu().numpy(), ref["gY0"], rtol=1e-13, atol=0)
    assert np.all(st.cpu().numpy() == 0)
