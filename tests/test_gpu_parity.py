"""CUDA path vs the CPU oracle on the same seeded inputs, through the C ABI.

Tolerances (from the requirements of the method): rates and Jacobian within 1e-12 relative to the size
of the terms that make them up (|x| + gross, the gross sizes are returned by the oracle); integrated
T and Y within 1e-8 relative for Y > 1e-12 on cells whose accepted/rejected step sequence matches the
oracle's.  An adaptive integrator can take a different decision where the error estimate is within
rounding of 1; such cells are counted, must be rare, and must still agree to the integration
tolerance.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle.oracle import Oracle  # noqa: E402
from paper_2311_14941_gb300 import chem, synth  # noqa: E402

MECHS = {"small": synth.mechanism_small, "mid": synth.mechanism_methane_sized, "large": synth.mechanism_large}
RTOL_RATES = 1e-12
RTOL_INT = 1e-8


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


_cache = {}


def mech(name):
    if name not in _cache:
        m = MECHS[name]()
        _cache[name] = (m, chem.create(m, 0), Oracle(m))
    return _cache[name]


def states(m, name):
    """Random states over the whole T range plus flame-like and special states."""
    F = synth.field_uniform_random(m, 40, seed=21, T_range=(320.0, 2900.0))
    T, p, Y = [F.T], [F.p], [F.Y]
    if name != "small":
        G = synth.field_bimodal_jet(m, 8, 8, seed=3)
        T.append(G.T); p.append(G.p); Y.append(G.Y)
    H = synth.field_igniting(m, 8, seed=5)
    T.append(H.T); p.append(H.p); Y.append(H.Y)
    # special: species absent, T at the NASA switch, high pressure
    Z = F.Y[:, :4].copy()
    Z[: m.n_species // 2] = 0.0
    Z /= Z.sum(axis=0)
    T.append(np.array([1500.0, 999.999, 1000.0, 2400.0])); p.append(np.array([1e5, 1e5, 3e5, 2e6])); Y.append(Z)
    return np.concatenate(T), np.concatenate(p), np.concatenate(Y, axis=1)


def to_dev(a, dev, dtype=torch.float64):
    return torch.tensor(np.ascontiguousarray(a), dtype=dtype, device=dev)


@pytest.mark.parametrize("name", list(MECHS))
def test_rates_parity(name, dev):
    m, h, o = mech(name)
    T, p, Y = states(m, name)
    N = T.shape[0]
    dT = torch.empty(N, dtype=torch.float64, device=dev)
    dY = torch.empty(m.n_species * N, dtype=torch.float64, device=dev)
    wd = torch.empty(m.n_species * N, dtype=torch.float64, device=dev)
    h.rates(to_dev(T, dev), to_dev(p, dev), to_dev(Y, dev), dT, dY, wd)
    torch.cuda.synchronize()
    dT, dY, wd = dT.cpu().numpy(), dY.cpu().numpy().reshape(m.n_species, N), wd.cpu().numpy().reshape(m.n_species, N)
    worst = 0.0
    for c in range(N):
        r = o.rhs(T[c], p[c], Y[:, c], want_gross=True)
        g = np.concatenate([[dT[c]], dY[:, c]])
        err = np.abs(g - r["f"]) / (np.abs(r["f"]) + r["gross"] + 1e-300)
        worst = max(worst, err.max())
        gw = r["gross"][1:] * (p[c] / (8.314462618 * T[c]) / np.sum(Y[:, c] / m.W)) / m.W
        assert np.all(np.abs(wd[:, c] - r["wdot"]) <= RTOL_RATES * (np.abs(r["wdot"]) + gw) + 1e-300)
    assert worst <= RTOL_RATES, worst


@pytest.mark.parametrize("name", list(MECHS))
def test_jacobian_parity(name, dev):
    m, h, o = mech(name)
    T, p, Y = states(m, name)
    N = T.shape[0]
    nnz = h.info["nnz_S"]
    S = torch.empty(nnz * N, dtype=torch.float64, device=dev)
    u = torch.empty(h.m * N, dtype=torch.float64, device=dev)
    v = torch.empty(h.m * N, dtype=torch.float64, device=dev)
    h.jacobian(to_dev(T, dev), to_dev(p, dev), to_dev(Y, dev), S, u, v)
    torch.cuda.synchronize()
    S = S.cpu().numpy().reshape(nnz, N)
    u = u.cpu().numpy().reshape(h.m, N)
    v = v.cpu().numpy().reshape(h.m, N)
    rp, ci = h.jacobian_pattern()
    worst = 0.0
    for c in range(N):
        Jg = np.outer(u[:, c], v[:, c])
        for r in range(h.m):
            Jg[r, ci[rp[r]:rp[r + 1]]] += S[rp[r]:rp[r + 1], c]
        J, G = o.jacobian(T[c], p[c], Y[:, c], want_gross=True)
        err = np.abs(Jg - J) / (np.abs(J) + G + 1e-300)
        worst = max(worst, err.max())
    assert worst <= RTOL_RATES, worst


def _integrate_gpu(h, F, dev, trace_cap=0, **kw):
    N = F.n_cells
    T = to_dev(F.T, dev)
    Y = to_dev(F.Y.reshape(-1), dev)
    hio = torch.zeros(N, dtype=torch.float64, device=dev)
    ns = torch.zeros(N, dtype=torch.int32, device=dev)
    st = torch.zeros(N, dtype=torch.int32, device=dev)
    tr = torch.zeros(trace_cap * N, dtype=torch.float64, device=dev) if trace_cap else None
    h.integrate(T, to_dev(F.p, dev), Y, to_dev(F.dt, dev), hio, ns, st, trace=tr, **kw)
    torch.cuda.synchronize()
    out = dict(T=T.cpu().numpy(), Y=Y.cpu().numpy().reshape(F.Y.shape), h=hio.cpu().numpy(),
               nsub=ns.cpu().numpy(), status=st.cpu().numpy())
    if trace_cap:
        out["trace"] = tr.cpu().numpy().reshape(trace_cap, N)
    return out


def _noise_floor(o, F, c, trace_col, method=0, tab_tol=0.0):
    """Sensitivity of the oracle's own result for cell c to a 1e-15 relative perturbation of its input
    (same step sequence): the floor below which two correct FP64 implementations cannot agree.
    Tabulated runs compare two independently built tables, each within tab_tol of the exact functions
    (their own coefficients; a temperature on an interval boundary may take either neighbour's
    polynomial): two such approximations agree to within the sum of their errors, not to rounding.  That
    part of the floor is the oracle's own tabulated-minus-exact result on the same steps."""
    hs = trace_col[trace_col > 0]
    y0 = o.state(F.T[c], F.Y[:, c])
    base = o.replay(y0, F.p[c], hs, method=method, tab_tol=tab_tol)
    rng = np.random.default_rng(c)
    sig = np.zeros_like(base)
    for _ in range(3):
        yp = y0 * (1.0 + 1e-15 * rng.standard_normal(y0.shape))
        sig = np.maximum(sig, np.abs(o.replay(yp, F.p[c], hs, method=method, tab_tol=tab_tol) - base))
    if tab_tol > 0:
        sig = np.maximum(sig, np.abs(base - o.replay(y0, F.p[c], hs, method=method)))
    return sig


def _compare_integration(o, g, r, F, max_flip_frac, method=0, tab_tol=0.0):
    """Cells with the same accept/reject sequence: every T and Y > 1e-12 within 1e-8 relative, or within
    10x the oracle's own rounding-propagation floor where that is larger (tiny species set by fast
    balances).  Cells whose sequence differs (a decision at err ~ 1 flipped by rounding): within
    10 rtol relative (10 atol absolute)."""
    assert np.array_equal(g["status"], r["status"]), (g["status"], r["status"])
    # Same sequence: identical accept/reject decisions and step sizes equal up to the rounding of the
    # error estimate (the last, clipped step dt - t inherits the rounding of t: dt-relative term).
    # Anything else -- a flipped decision, or a rejection taken through the non-finite branch (h/10)
    # on one side and the error branch (h/5) on the other -- is a different sequence.
    hr = np.abs(r["trace"])
    hdiff = np.abs(np.abs(g["trace"]) - hr) / (hr + 1e-9 * F.dt[None, :])
    same = np.all(np.sign(g["trace"]) == np.sign(r["trace"]), axis=0) & np.all(hdiff <= 1e-4, axis=0)
    flips = np.where(~same)[0]
    assert len(flips) <= max(1, int(max_flip_frac * F.n_cells)), (len(flips), F.n_cells)
    hdiff = hdiff[:, same]
    yg = np.vstack([g["T"][None, :], g["Y"]])
    yr = np.vstack([r["T"][None, :], r["Y"]])
    big = np.abs(yr) > 1e-12
    big[0] = True
    d = np.abs(yg - yr)
    ok = (d <= RTOL_INT * np.abs(yr)) | ~big
    floor_cells = 0
    worst = 0.0
    for c in np.where(same & ~np.all(ok, axis=0))[0]:
        sig = _noise_floor(o, F, c, r["trace"][:, c], method, tab_tol)
        bad = big[:, c] & (d[:, c] > np.maximum(RTOL_INT * np.abs(yr[:, c]), 10.0 * sig))
        assert not bad.any(), (c, np.where(bad)[0], d[bad, c], yr[bad, c], sig[bad])
        floor_cells += 1
    rel = np.where(big, d / np.where(big, np.abs(yr), 1.0), 0.0)
    worst = rel[:, same & np.all(ok, axis=0)].max(initial=0.0)
    for c in flips:
        assert np.all(d[:, c] <= 10 * 1e-6 * np.abs(yr[:, c]) + 10 * 1e-12), c
    print(f"cells {F.n_cells}: same sequence {int(same.sum())} (max step-size drift {hdiff.max():.1e}), "
          f"flips {len(flips)}, "
          f"within 1e-8 everywhere {int((same & np.all(ok, axis=0)).sum())} (worst {worst:.2e}), "
          f"at the rounding floor {floor_cells}")
    return len(flips)


@pytest.mark.parametrize("wpc,method,cpw,mode", [(1, 0, 1, 0), (2, 0, 1, 0), (1, 1, 1, 0), (1, 2, 1, 0), (2, 2, 1, 0),
                                              (1, 0, 2, 0), (1, 0, 2, 1), (1, 2, 2, 1)])
def test_integrate_parity_small_full_config(dev, wpc, method, cpw, mode):
    """1024 cells, 10 species / 27 reactions, p = 1 atm, T ~ U(900, 2200) K, Dirichlet Y, dt = 1e-5 s;
    one or two warps per cell, or two cells per warp (plain and sorted-queue launches); RODAS3 (method
    0), ROS2 (method 1) or RODAS4 (method 2)."""
    m, h, o = mech("small")
    F = synth.field_uniform_random(m, 1024, seed=1)
    r = o.integrate_batch(F.T, F.p, F.Y, F.dt, trace_cap=8000, method=method)
    g = _integrate_gpu(h, F, dev, trace_cap=8000, warps_per_cell=wpc, method=method, cells_per_warp=cpw, mode=mode)
    _compare_integration(o, g, r, F, 0.02, method)
    assert np.all(g["status"] == 0)


@pytest.mark.parametrize("wpc,method", [(1, 0), (2, 0), (1, 1), (1, 2)])
def test_integrate_parity_methane_sized_sample(dev, wpc, method):
    """120 cells of the bimodal jet field (cold, burnt and mixing-layer cells), 53/325 mechanism; one or
    two warps per cell; RODAS3, ROS2 or RODAS4."""
    m, h, o = mech("mid")
    F = synth.field_bimodal_jet(m, 256, 256, seed=2)
    rng = np.random.default_rng(7)
    idx = np.sort(np.concatenate([rng.choice(np.where(F.kind == k)[0], 40, replace=False) for k in (0, 1, 2)]))
    S = F.subset(idx)
    r = o.integrate_batch(S.T, S.p, S.Y, S.dt, trace_cap=4000, method=method)
    g = _integrate_gpu(h, S, dev, trace_cap=4000, warps_per_cell=wpc, method=method)
    _compare_integration(o, g, r, S, 0.03, method)


@pytest.mark.parametrize("wpc", [1, 2])
def test_integrate_parity_large_sample(dev, wpc):
    """16 cells of the 150/1000 mechanism with LTS-like dt in 1e-6..1e-4 s; one or two warps per cell."""
    m, h, o = mech("large")
    F = synth.field_bimodal_jet(m, 16, 16, seed=5, dt_range=(1e-6, 1e-4))
    S = F.subset(np.arange(0, 256, 16))
    r = o.integrate_batch(S.T, S.p, S.Y, S.dt, trace_cap=2000)
    g = _integrate_gpu(h, S, dev, trace_cap=2000, warps_per_cell=wpc)
    _compare_integration(o, g, r, S, 0.07)


def test_integrate_rejects_unknown_method(dev):
    m, h, o = mech("small")
    F = synth.field_uniform_random(m, 4, seed=4)
    for bad in (-1, 3):
        with pytest.raises(chem.ChemError):
            _integrate_gpu(h, F, dev, method=bad)


def test_integrate_edge_cases(dev):
    """Empty batch, a single cell, a ragged count, bad inputs, dt = 0 and the substep cap."""
    m, h, o = mech("small")
    F = synth.field_uniform_random(m, 37, seed=4)
    e = torch.empty(0, dtype=torch.float64, device=dev)
    ei = torch.empty(0, dtype=torch.int32, device=dev)
    h.integrate(e, e, e, e, e, ei, ei)          # N = 0 is a no-op
    one = F.subset([5])
    g = _integrate_gpu(h, one, dev)
    r = o.integrate_batch(one.T, one.p, one.Y, one.dt)
    assert g["nsub"][0] == r["nsub"][0] and abs(g["T"][0] - r["T"][0]) <= 1e-8 * r["T"][0]
    B = F.subset(np.arange(37))
    B.T[3] = -10.0
    B.Y[2, 4] = np.nan
    B.dt[5] = -1e-6
    B.p[6] = 0.0
    B.dt[7] = 0.0
    g = _integrate_gpu(h, B, dev)
    r = o.integrate_batch(B.T, B.p, B.Y, B.dt)
    assert list(g["status"][3:7]) == [4, 4, 4, 4] and np.array_equal(g["status"], r["status"])
    assert g["nsub"][7] == 0 and g["T"][7] == B.T[7]
    keep = np.setdiff1d(np.arange(37), [3, 4, 5, 6])
    assert np.all(np.abs(g["T"][keep] - r["T"][keep]) <= 1e-8 * np.abs(r["T"][keep]) + 1e-6 * (g["nsub"][keep] != r["nsub"][keep]) * r["T"][keep])
    g = _integrate_gpu(h, F.subset(np.arange(8)), dev, max_substeps=3)
    r = o.integrate_batch(F.T[:8], F.p[:8], F.Y[:, :8], F.dt[:8], max_steps=3)
    assert np.all(g["status"] == 1) and np.array_equal(g["status"], r["status"])
    assert np.all(g["nsub"] == 3)
    assert np.allclose(g["T"], r["T"], rtol=1e-10)


def _lts_regime_cells(m):
    """224 cells of the 262,144-cell LTS mix (per-cell dt log-uniform 1e-7..1e-3 s), stratified so that
    cold, burnt and igniting cells each come with dt above and below 1e-4 s, plus 16 igniting cells of
    the adjoint workload (T0 1000-1400 K, p 1-10 atm) over dt = 1e-3 s, which take 500 to 3,500 steps."""
    F = synth.field_lts_mix(m, 262144, seed=3)
    rng = np.random.default_rng(23)
    big = F.dt > 1e-4
    pick = []
    for k, n in ((0, 96), (1, 64), (3, 64)):
        pick += list(rng.choice(np.where((F.kind == k) & ~big)[0], n // 2, replace=False))
        pick += list(rng.choice(np.where((F.kind == k) & big)[0], n - n // 2, replace=False))
    S = F.subset(np.sort(np.array(pick)))
    G = synth.field_igniting(m, 4096, seed=4, dt=1e-3)
    Sg = G.subset(np.sort(rng.choice(4096, 16, replace=False)))
    return synth.Field(np.concatenate([S.T, Sg.T]), np.concatenate([S.p, Sg.p]), np.concatenate([S.Y, Sg.Y], axis=1),
                       np.concatenate([S.dt, Sg.dt]), np.concatenate([S.kind, Sg.kind]))


@pytest.mark.parametrize("wpc", [1, 2])
def test_sorted_queue_parity_long_dt_regime(dev, wpc):
    """The sorted work queue (mode 1) against the oracle in the regime of the LTS and adjoint workloads:
    dt up to 1e-3 s, cold, burnt and igniting cells, with a previous-step cost key that reorders them;
    one and two warps per cell; same trace-matched criteria as the other integration tests."""
    m, h, o = mech("mid")
    F = _lts_regime_cells(m)
    cap = 4000
    r = o.integrate_batch(F.T, F.p, F.Y, F.dt, trace_cap=cap)
    assert r["nsub"].max() < cap and r["nsub"].max() > 2000
    N = F.n_cells
    key = np.random.default_rng(5).integers(0, 3000, N).astype(np.int32)
    T = to_dev(F.T, dev)
    Y = to_dev(F.Y.reshape(-1), dev)
    hio = torch.zeros(N, dtype=torch.float64, device=dev)
    ns = torch.tensor(key, device=dev)
    st = torch.zeros(N, dtype=torch.int32, device=dev)
    tr = torch.zeros(cap * N, dtype=torch.float64, device=dev)
    h.integrate(T, to_dev(F.p, dev), Y, to_dev(F.dt, dev), hio, ns, st, trace=tr, mode=1, warps_per_cell=wpc,
                chunk=2)
    torch.cuda.synchronize()
    g = dict(T=T.cpu().numpy(), Y=Y.cpu().numpy().reshape(F.Y.shape), h=hio.cpu().numpy(), nsub=ns.cpu().numpy(),
             status=st.cpu().numpy(), trace=tr.cpu().numpy().reshape(cap, N))
    assert np.all(g["status"] == 0)
    _compare_integration(o, g, r, F, 0.1)


@pytest.mark.parametrize("name,mode", [("small", 0), ("mid", 1)])
def test_tabulated_parity_against_the_oracles_tables(dev, name, mode):
    """Tabulated temperature functions (tolerance 1e-10): the GPU's tables (built by the library) against
    the oracle's own tables, trace-matched as above, on the small mechanism's 1024-cell field and a jet
    and LTS sample of the methane-sized one; and the tabulated GPU result stays within 1e-6 of the
    exact GPU result.  The two sides build their tables independently (the same nodes and degrees,
    their own Chebyshev-to-power conversion), so tabulated values agree to about 1e-14 relative rather
    than to the last bit; the rounding floor of a tiny species includes that (see _noise_floor)."""
    m, h, o = mech(name)
    if name == "small":
        F = synth.field_uniform_random(m, 1024, seed=1)
    else:
        G = synth.field_bimodal_jet(m, 256, 256, seed=2)
        rng = np.random.default_rng(8)
        idx = np.sort(np.concatenate([rng.choice(np.where(G.kind == k)[0], 30, replace=False) for k in (0, 1, 2)]))
        F = G.subset(idx)
    r = o.integrate_batch(F.T, F.p, F.Y, F.dt, trace_cap=4000, tab_tol=1e-10)
    g = _integrate_gpu(h, F, dev, trace_cap=4000, tabulate=1, tab_tol=1e-10, mode=mode)
    _compare_integration(o, g, r, F, 0.03, tab_tol=1e-10)
    e = _integrate_gpu(h, F, dev, mode=mode)
    same = e["nsub"] == g["nsub"]
    assert same.mean() > 0.9 and np.any(e["T"] != g["T"])
    assert np.max(np.abs(e["T"][same] - g["T"][same]) / e["T"][same]) < 1e-6


def test_tabulated_options_are_checked(dev):
    m, h, o = mech("small")
    F = synth.field_uniform_random(m, 8, seed=2)
    for kw in (dict(tabulate=2), dict(tabulate=1, tab_tol=1.5), dict(tabulate=1, tab_tol=-1.0)):
        with pytest.raises(chem.ChemError):
            _integrate_gpu(h, F, dev, **kw)


# ------------------------------------------------------------------ mechanism-specialised kernels
_spec = {}


def spec_handle(name):
    """A handle of its own with the run-time compiled kernels (the cached handles above stay generic)."""
    if name not in _spec:
        h = chem.create(MECHS[name](), 0)
        h.specialize()
        _spec[name] = h
    return _spec[name]


def _spec_field(m, name):
    if name == "small":
        return synth.field_uniform_random(m, 1024, seed=1), 8000, 0.02
    if name == "mid":
        G = synth.field_bimodal_jet(m, 256, 256, seed=2)
        rng = np.random.default_rng(9)
        idx = np.sort(np.concatenate([rng.choice(np.where(G.kind == k)[0], 40, replace=False) for k in (0, 1, 2)]))
        return G.subset(idx), 4000, 0.03
    G = synth.field_bimodal_jet(m, 16, 16, seed=5, dt_range=(1e-6, 1e-4))
    return G.subset(np.arange(0, 256, 16)), 2000, 0.07


@pytest.mark.parametrize("name,mode", [("small", 0), ("small", 1), ("mid", 1), ("large", 0)])
def test_specialized_kernels_parity(dev, name, mode):
    """Mechanism-specialised one-warp kernels (sizes and shared-memory offsets compiled in at run time)
    against the oracle, trace-matched as above, on the three mechanisms (plain and sorted-queue form); and
    against the library's own one-warp kernels on the same inputs: the same step counts on almost every
    cell, the same results there to the integration tolerance."""
    m, _, o = mech(name)
    h = spec_handle(name)
    F, cap, flips = _spec_field(m, name)
    r = o.integrate_batch(F.T, F.p, F.Y, F.dt, trace_cap=cap)
    g = _integrate_gpu(h, F, dev, trace_cap=cap, warps_per_cell=1, mode=mode, specialized=1)
    _compare_integration(o, g, r, F, flips)
    e = _integrate_gpu(h, F, dev, warps_per_cell=1, mode=mode)
    same = e["nsub"] == g["nsub"]
    assert same.mean() >= 0.95, same.mean()
    assert np.max(np.abs(e["T"][same] - g["T"][same]) / e["T"][same]) <= RTOL_INT
    print(f"{name}: bit-identical to the library's kernels on {int(np.sum(e['T'] == g['T']))} of {F.n_cells} cells")


def test_specialized_options_are_checked(dev):
    m, plain_h, _ = mech("small")
    F = synth.field_uniform_random(m, 8, seed=2)
    with pytest.raises(chem.ChemError):                      # never specialised
        _integrate_gpu(plain_h, F, dev, specialized=1)
    h = spec_handle("small")
    for kw in (dict(specialized=2), dict(specialized=1, warps_per_cell=2), dict(specialized=1, cells_per_warp=2)):
        with pytest.raises(chem.ChemError):
            _integrate_gpu(h, F, dev, **kw)
    assert h.specialize() == 0.0                             # a second call does nothing
