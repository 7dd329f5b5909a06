"""Zonal reference-cell mapping (Sec. 2.5: the chemistry solution of low-reactivity cells is mapped from
a reference cell).  CPU: the oracle's reading pinned to closed forms and hand-counted zones.  GPU:
chem_integrate_mapped against the oracle (zones bit for bit, values within the integration
tolerance) and against plain chem_integrate when nothing is mapped."""
import math

import numpy as np
import pytest

from oracle import zonal
from oracle.oracle import Oracle
from paper_2311_14941_gb300 import synth
from tests import tinymech as tm

P0 = 101325.0


def _ab_mech(k):
    th = tm.const_cp_thermo(3.5)
    return tm.build([0.03, 0.03], [(th, th), (th, th)], [dict(re=[(0, 1)], pr=[(1, 1)], A=k, rev=0)])


def test_mapped_member_takes_the_reference_change_closed_form():
    """A -> B, isothermal: the reference decays as Y_A,r exp(-k dt); a member of its zone receives
    Y_A,c + Y_A,r (exp(-k dt) - 1), not its own exact decay."""
    k, dt = 2.0e5, 1e-5
    o = Oracle(_ab_mech(k))
    YA = np.array([0.90, 0.93, 0.97, 0.50])
    Y = np.vstack([YA, 1.0 - YA])
    T = np.full(4, 1200.0)
    out = zonal.integrate_mapped(o, T, np.full(4, P0), Y, np.full(4, dt),
                                 dict(T_max=1500.0, dT=100.0, species=[0], dY=[0.1]), rtol=1e-10, atol=1e-15)
    assert out["ref"].tolist() == [0, 0, 0, 3]          # 0.90, 0.93 and 0.97 share the bin [0.9, 1.0)
    assert out["n_integrated"] == 2
    e = math.exp(-k * dt)
    for c in (0, 3):
        assert out["Y"][0, c] == pytest.approx(YA[c] * e, rel=1e-8)
    for c in (1, 2):
        assert out["Y"][0, c] == pytest.approx(YA[c] + YA[0] * (e - 1.0), rel=1e-8)
        assert abs(out["Y"][0, c] - YA[c] * e) > 1e-4    # really mapped, not integrated
        assert out["nsub"][c] == 0 and out["status"][c] == 0
    assert np.allclose(out["Y"].sum(axis=0), 1.0, atol=1e-14)
    assert np.all(out["T"] == 1200.0)


def test_zones_by_hand():
    """Bin edges, T_max, pressure and dt separate zones; identical cells share one; the lowest index leads."""
    n = 3
    Y = np.tile(np.array([[0.2], [0.3], [0.5]]), (1, 9))
    T = np.array([450.0, 460.0, 399.999, 400.0, 700.0, 450.0, 450.0, 455.0, 450.0])
    p = np.array([P0, P0, P0, P0, P0, 2 * P0, P0, P0, P0])
    dt = np.array([1e-5, 1e-5, 1e-5, 1e-5, 1e-5, 1e-5, 2e-5, 1e-5, 1e-5])
    Y[1, 8] = 0.36                                     # another Y_1 bin (dY = 0.05)
    Y[2, 7] = 0.99                                     # species 2 is not in the key
    ref = zonal.references(T, p, Y, dt, T_max=600.0, dT=100.0, species=[1], dY=[0.05])
    # 450, 460 and 400 share floor(T/100) = 4; 399.999 is in bin 3; 700 >= T_max; 2p and 2dt stand alone;
    # 455 differs only in species 2, which is not in the key; Y_1 = 0.36 is in another bin
    assert ref.tolist() == [0, 0, 2, 0, 4, 5, 6, 0, 8]
    none = zonal.references(T, p, Y, dt, T_max=0.0, dT=100.0)
    assert np.array_equal(none, np.arange(9))
    # non-finite key values and quotients beyond 2^62 are not candidates
    T2 = np.array([450.0, 450.0, 450.0])
    Y2 = np.array([[0.2, 0.2, np.nan], [0.3, 0.3, 0.3], [0.5, 0.5, 0.5]])
    assert zonal.references(T2, np.full(3, P0), Y2, np.full(3, 1e-5), 600.0, 1e-300, [1], [1e-300]).tolist() == \
        [0, 1, 2]
    assert zonal.references(T2, np.full(3, P0), Y2, np.full(3, 1e-5), 600.0, 100.0, [0], [0.1]).tolist() == \
        [0, 0, 2]
    assert n == Y.shape[0]


def test_no_mapping_is_plain_integration():
    m = synth.mechanism_small()
    o = Oracle(m)
    F = synth.field_uniform_random(m, 12, seed=3)
    a = zonal.integrate_mapped(o, F.T, F.p, F.Y, F.dt, None, nthreads=1)
    b = o.integrate_batch(F.T, F.p, F.Y, F.dt, 1e-6, 1e-12, nthreads=1)
    assert np.array_equal(a["T"], b["T"]) and np.array_equal(a["Y"], b["Y"]) and a["n_integrated"] == 12
    assert np.array_equal(a["ref"], np.arange(12))


# ----------------------------------------------------------------------------------------------- GPU
def _gpu_field(F, dev):
    import torch
    t = lambda a, dt=torch.float64: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=dev)
    N = F.n_cells
    return dict(T=t(F.T), p=t(F.p), Y=t(F.Y.reshape(-1)), dt=t(F.dt), h=t(np.zeros(N)),
                ns=t(np.zeros(N), torch.int32), st=t(np.zeros(N), torch.int32), ref=t(np.zeros(N), torch.int32))


def _cold_key(m, F):
    """The two species whose mass fractions vary most over the cold cells (the fuel/air mixture)."""
    cold = F.T < 700.0
    sp = np.argsort(-F.Y[:, cold].std(axis=1))[:2]
    return dict(T_max=700.0, dT=20.0, species=[int(s) for s in sp], dY=[0.02, 0.02])


@pytest.fixture(scope="module")
def dev():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    return torch.device("cuda", 0)


@pytest.mark.gpu
@pytest.mark.parametrize("mode", [0, 1])
def test_mapped_integration_matches_oracle(dev, mode):
    """4096 cells of the bimodal jet field, 10/27 mechanism, dt 1e-5 s: cold cells (< 700 K) mapped by
    (T, two key species).  Zones bit for bit; integrated cells bit-identical to chem_integrate and within
    the integration tolerance of the oracle; members exactly T_c + (T_ref(dt) - T_ref(0)) (and Y)."""
    import torch
    from paper_2311_14941_gb300 import chem
    m = synth.mechanism_small()
    F = synth.field_bimodal_jet(m, 64, 64, seed=4)
    mp = _cold_key(m, F)
    h = chem.create(m, 0)
    g = _gpu_field(F, dev)
    M = h.integrate_mapped(g["T"], g["p"], g["Y"], g["dt"], g["h"], g["ns"], g["st"], g["ref"], mp, mode=mode)
    torch.cuda.synchronize()
    N, n = F.n_cells, m.n_species
    ref = g["ref"].cpu().numpy()
    want = zonal.references(F.T, F.p, F.Y, F.dt, mp["T_max"], mp["dT"], mp["species"], mp["dY"])
    assert np.array_equal(ref, want)
    integ = ref == np.arange(N)
    assert M == int(integ.sum()) and M < 0.75 * N           # a good share of the cold cells is mapped
    Tg, Yg = g["T"].cpu().numpy(), g["Y"].cpu().numpy().reshape(n, N)
    nsg, stg, hg = g["ns"].cpu().numpy(), g["st"].cpu().numpy(), g["h"].cpu().numpy()
    # integrated cells: bit for bit the plain chem_integrate results
    q = _gpu_field(F, dev)
    h.integrate(q["T"], q["p"], q["Y"], q["dt"], q["h"], q["ns"], q["st"], mode=mode)
    torch.cuda.synchronize()
    Tq, Yq = q["T"].cpu().numpy(), q["Y"].cpu().numpy().reshape(n, N)
    assert np.array_equal(Tg[integ], Tq[integ]) and np.array_equal(Yg[:, integ], Yq[:, integ])
    assert np.array_equal(nsg[integ], q["ns"].cpu().numpy()[integ])
    assert np.array_equal(stg[integ], q["st"].cpu().numpy()[integ])
    # members: the reference's change added, in the same floating-point order
    mem = np.flatnonzero(~integ)
    r = ref[mem]
    assert np.array_equal(Tg[mem], F.T[mem] + (Tg[r] - F.T[r]))
    assert np.array_equal(Yg[:, mem], F.Y[:, mem] + (Yg[:, r] - F.Y[:, r]))
    assert np.all(nsg[mem] == 0) and np.array_equal(stg[mem], stg[r]) and np.all(hg[mem] == 0.0)
    # against the oracle's mapped integration
    o = Oracle(m)
    want = zonal.integrate_mapped(o, F.T, F.p, F.Y, F.dt, mp)
    assert want["n_integrated"] == M
    assert np.array_equal(stg, want["status"])
    y_g = np.vstack([Tg[None, :], Yg])
    y_o = np.vstack([want["T"][None, :], want["Y"]])
    scale = np.abs(y_o) + np.abs(np.vstack([want["T"][None, :], want["Y"]])[:, want["ref"]])
    d = np.abs(y_g - y_o)
    big = scale > 1e-12
    assert np.all(d[big] <= 1e-5 * scale[big] + 1e-11)                       # every cell: 10 rtol
    tight = np.all((d <= 1e-8 * scale) | ~big, axis=0)
    assert tight.mean() > 0.97, tight.mean()                                 # most: the 1e-8 bar
    print(f"mapped {N - M} of {N} cells; {tight.mean():.4f} of cells within 1e-8")


@pytest.mark.gpu
def test_no_mapping_equals_chem_integrate(dev):
    import torch
    from paper_2311_14941_gb300 import chem
    m = synth.mechanism_small()
    F = synth.field_uniform_random(m, 777, seed=6)
    h = chem.create(m, 0)
    a, b = _gpu_field(F, dev), _gpu_field(F, dev)
    M = h.integrate_mapped(a["T"], a["p"], a["Y"], a["dt"], a["h"], a["ns"], a["st"], a["ref"], None, mode=1)
    h.integrate(b["T"], b["p"], b["Y"], b["dt"], b["h"], b["ns"], b["st"], mode=1)
    torch.cuda.synchronize()
    assert M == 777
    assert np.array_equal(a["ref"].cpu().numpy(), np.arange(777))
    for k in ("T", "Y", "h", "ns", "st"):
        assert torch.equal(a[k], b[k]), k


@pytest.mark.gpu
def test_mapping_rejects_bad_options(dev):
    from paper_2311_14941_gb300 import chem
    m = synth.mechanism_small()
    F = synth.field_uniform_random(m, 8, seed=6)
    h = chem.create(m, 0)
    g = _gpu_field(F, dev)
    args = (g["T"], g["p"], g["Y"], g["dt"], g["h"], g["ns"], g["st"], g["ref"])
    for bad in (dict(T_max=700.0, dT=0.0), dict(T_max=700.0, dT=-1.0), dict(T_max=float("nan"), dT=10.0),
                dict(T_max=700.0, dT=10.0, species=[0, 0], dY=[0.1, 0.1]),
                dict(T_max=700.0, dT=10.0, species=[m.n_species], dY=[0.1]),
                dict(T_max=700.0, dT=10.0, species=[1], dY=[0.0])):
        with pytest.raises(chem.ChemError) as ei:
            h.integrate_mapped(*args, bad)
        assert "status 1" in str(ei.value)
    assert h.integrate_mapped(*args, dict(T_max=-1.0, dT=10.0)) == 8      # nothing below T_max
