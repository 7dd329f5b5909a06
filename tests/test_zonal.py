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
