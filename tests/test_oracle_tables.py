"""Pins of the oracle's tabulated temperature functions (the opt-in approximation of Sec. 2.5's
"optimal-degree interpolation of costly thermodynamic functions").

What the oracle tabulates: exp(g_k) and exp(-g_k) of every species (g_k = h_k/(Ru T) - s_k/Ru), every
reaction's forward rate coefficient (the high-pressure limit of a fall-off reaction), and each fall-off
reaction's Troe centre F_cent, as piecewise polynomials in u = 1/T over 250 K <= T < 4000 K (640 equal intervals of u),
one polynomial degree per class of functions, the smallest meeting the relative tolerance.

Pinned here without the oracle's table code:
- every tabulated value is within the tolerance of the exact function, which numpy evaluates from the
  description (Arrhenius and Troe forms) or from the oracle's NASA-7 routine (pinned elsewhere), at
  random temperatures, including the interval ends and T = 1000 K;
- the degree of a class is the smallest that meets the tolerance: numpy's own Chebyshev interpolation at
  the same points, with one degree less, misses it on some interval;
- outside the range the exact functions are used;
- integrating with the tables stays within 1e-8 relative of the exact integration (tolerance 1e-10).
"""
import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2311_14941_gb300 import synth

RU = 8.314462618
TOL = 1e-10


def exact(m, o, cls, f, T):
    T = float(T)
    if cls in (0, 1):
        cp, hRT, sR = o.thermo(T)
        g = hRT[f] - sR[f]
        return np.exp(g) if cls == 0 else np.exp(-g)
    troe = np.where(np.asarray(m.rtype) == 2)[0]
    if cls == 2:
        return m.A[f] * T ** m.b[f] * np.exp(-m.Ea[f] / (RU * T))
    r = troe[f]
    a, T3, T1, T2 = np.asarray(m.troe).reshape(-1, 4)[r]
    return (1 - a) * np.exp(-T / T3) + a * np.exp(-T / T1) + (np.exp(-T2 / T) if T2 > 0 else 0.0)


def n_functions(m, cls):
    nt = int(np.sum(np.asarray(m.rtype) == 2))
    return [m.n_species, m.n_species, m.n_reactions, nt][cls]


@pytest.mark.parametrize("mk", [synth.mechanism_small, synth.mechanism_methane_sized])
def test_tabulated_values_within_tolerance(mk):
    m = mk()
    o = Oracle(m)
    _, deg, ni, rng = o.tab_build(TOL)
    assert deg.min() >= 1 and deg.max() <= 8 and ni == 640
    Tlo, Thi, ulo, du = rng
    gen = np.random.default_rng(4)
    # random temperatures, interval ends and the NASA-7 switch
    Ts = np.concatenate([gen.uniform(Tlo, Thi, 40), 1.0 / (ulo + du * gen.integers(1, ni, 8)), [1000.0, Tlo]])
    worst = 0.0
    for cls in range(4):
        nf = n_functions(m, cls)
        for f in gen.choice(nf, min(nf, 12), replace=False) if nf else []:
            for T in Ts:
                ex = exact(m, o, cls, int(f), T)
                tv = o.tab_eval(TOL, cls, int(f), T)
                rel = abs(tv - ex) / abs(ex)
                worst = max(worst, rel)
                # the exact reference here differs from the oracle's own (pow vs exp-log) by a few ulp
                assert rel <= TOL * (1 + 1e-3) + 1e-14, (cls, f, T, rel)
    assert worst > 1e-14   # the values are interpolated, not exact


def test_degree_is_the_smallest_meeting_the_tolerance():
    """numpy's Chebyshev interpolation at the same points, for the forward rate coefficients and the
    species factors of the small mechanism: the oracle's degree meets the tolerance, one less does not."""
    m = synth.mechanism_small()
    o = Oracle(m)
    _, deg, ni, rng = o.tab_build(TOL)
    Tlo, Thi, ulo, du = rng
    C = np.polynomial.chebyshev

    def worst(cls, d):
        w = 0.0
        for f in range(n_functions(m, cls)):
            for j in range(ni):
                u0 = ulo + j * du
                fn = lambda tau: np.array([exact(m, o, cls, f, 1.0 / (u0 + 0.5 * (t + 1) * du)) for t in tau])
                c = C.chebinterpolate(fn, d)
                tau = np.linspace(-1, 1, 17)
                ex = fn(tau)
                w = max(w, np.max(np.abs(C.chebval(tau, c) - ex) / np.abs(ex)))
        return w

    for cls in (2, 3):
        d = int(deg[cls])
        assert worst(cls, d) <= TOL * 1.01
        assert worst(cls, d - 1) > TOL


def test_outside_the_range_the_exact_functions():
    m = synth.mechanism_small()
    o = Oracle(m)
    for T in (200.0, 4000.0, 5200.0):
        for cls, f in ((0, 2), (2, 5)):
            assert o.tab_eval(TOL, cls, f, T) == pytest.approx(exact(m, o, cls, f, T), rel=1e-14)


def test_tabulated_integration_stays_close_to_exact():
    m = synth.mechanism_small()
    o = Oracle(m)
    F = synth.field_uniform_random(m, 48, seed=6)
    a = o.integrate_batch(F.T, F.p, F.Y, F.dt)
    b = o.integrate_batch(F.T, F.p, F.Y, F.dt, tab_tol=TOL)
    assert np.all(a["status"] == 0) and np.all(b["status"] == 0)
    same = a["nsub"] == b["nsub"]
    assert same.mean() > 0.9
    assert np.max(np.abs(a["T"][same] - b["T"][same]) / a["T"][same]) <= 1e-8
    big = np.abs(a["Y"]) > 1e-10
    rel = np.abs(a["Y"] - b["Y"]) / np.where(big, np.abs(a["Y"]), 1.0)
    assert np.max(rel[:, same][big[:, same]]) <= 1e-6
    assert np.any(a["T"] != b["T"])   # the tables were used
