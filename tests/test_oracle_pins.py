"""Pins of the CPU oracle to facts outside itself: closed forms, invariants, an independent ODE library,
complex-step derivatives, and the published order conditions of the Rosenbrock method.

Each test names what it pins.  None of them re-types an oracle formula: they check properties that a
dropped term, a wrong sign or index, or a transposed operand would break.
"""
import math

import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2311_14941_gb300 import synth
from tests import tinymech as tm

RU = 8.314462618
P0 = 101325.0


@pytest.fixture(scope="module")
def small():
    m = synth.mechanism_small()
    return m, Oracle(m)


@pytest.fixture(scope="module")
def mid():
    m = synth.mechanism_methane_sized()
    return m, Oracle(m)


# ------------------------------------------------------------------------------------ method tableau
def test_rodas3_order_conditions_and_L_stability(small):
    """RODAS3 (Sandu et al. 1997): order 3 with an order-2 embedded pair, stiffly accurate, R(-inf) = 0."""
    t = small[1].tableau()
    s, g = t["s"], t["gamma"]
    a, gm, b, bh = t["alpha"][:s, :s], t["gam"][:s, :s], t["b"][:s], t["bhat"][:s]
    beta_m = a + gm                       # strictly lower
    beta = beta_m.sum(axis=1)
    alp = a.sum(axis=1)
    assert abs(b.sum() - 1) < 1e-15
    assert abs(b @ beta - (0.5 - g)) < 1e-15
    assert abs(b @ alp ** 2 - 1.0 / 3.0) < 1e-15
    assert abs(b @ (beta_m @ beta) - (1.0 / 6.0 - g + g * g)) < 1e-15
    # embedded method: order 2
    assert abs(bh.sum() - 1) < 1e-15
    assert abs(bh @ beta - (0.5 - g)) < 1e-15
    # stiffly accurate: last row of beta equals b, last weight equals gamma
    assert np.allclose(beta_m[s - 1, : s - 1], b[: s - 1], atol=1e-15) and abs(b[s - 1] - g) < 1e-15
    # linear stability function R(z) = 1 + z b^T (I - z B)^-1 1 with B = alpha + Gamma (diag gamma)
    B = beta_m + g * np.eye(s)

    def R(z):
        return 1 + z * b @ np.linalg.solve(np.eye(s) - z * B, np.ones(s))

    assert abs(1 - b @ np.linalg.solve(B, np.ones(s))) < 1e-14          # R(inf) = 0
    assert abs(R(-1e12)) < 1e-10
    assert max(abs(R(1j * y)) for y in np.logspace(-3, 6, 200)) <= 1 + 1e-12   # A-stable on the imaginary axis
    assert max(abs(R(x)) for x in -np.logspace(-3, 8, 200)) <= 1 + 1e-12


def test_ros2_order_conditions_and_L_stability(small):
    """ROS2 (Verwer et al. 1999): order 2 with a first-order embedded solution, gamma = 1 + 1/sqrt(2),
    R(-inf) = 0 (L-stable); the controller uses err^(-1/2)."""
    t = small[1].tableau(method=1)
    s, g = t["s"], t["gamma"]
    assert s == 2 and t["err_order"] == 2 and small[1].tableau()["err_order"] == 3
    assert abs(g - (1 + 1 / math.sqrt(2))) < 1e-15
    a, gm, b, bh = t["alpha"][:s, :s], t["gam"][:s, :s], t["b"][:s], t["bhat"][:s]
    beta_m = a + gm
    beta = beta_m.sum(axis=1)
    assert abs(b.sum() - 1) < 1e-15
    assert abs(b @ beta - (0.5 - g)) < 1e-15
    # the third-order condition fails (order exactly 2)
    assert abs(b @ a.sum(axis=1) ** 2 - 1.0 / 3.0) > 0.1
    assert abs(bh.sum() - 1) < 1e-15 and abs(bh @ beta - (0.5 - g)) > 0.1   # embedded: order 1
    B = beta_m + g * np.eye(s)

    def R(z):
        return 1 + z * b @ np.linalg.solve(np.eye(s) - z * B, np.ones(s))

    assert abs(1 - b @ np.linalg.solve(B, np.ones(s))) < 1e-14          # R(inf) = 0
    assert max(abs(R(1j * y)) for y in np.logspace(-3, 6, 200)) <= 1 + 1e-12
    assert max(abs(R(x)) for x in -np.logspace(-3, 8, 200)) <= 1 + 1e-12


def _rosenbrock_conditions(b, a, gm, g, order):
    """Residuals of the Rosenbrock order conditions up to `order` (Hairer and Wanner, Sec. VI.7, with
    beta_ij = alpha_ij + gamma_ij and beta'_i = sum_{j<i} beta_ij) for weights b."""
    bm = a + gm
    be = bm.sum(axis=1)
    al = a.sum(axis=1)
    r = [b.sum() - 1, b @ be - (0.5 - g)]
    if order >= 3:
        r += [b @ al ** 2 - 1.0 / 3.0, b @ (bm @ be) - (1.0 / 6.0 - g + g * g)]
    if order >= 4:
        r += [b @ al ** 3 - 0.25, b @ (al * (a @ be)) - (1.0 / 8.0 - g / 3.0), b @ (bm @ al ** 2) - (1.0 / 12.0 - g / 3.0),
              b @ (bm @ (bm @ be)) - (1.0 / 24.0 - g / 2.0 + 1.5 * g * g - g ** 3)]
    return np.array(r)


def test_rodas4_order_conditions_and_L_stability(small):
    """RODAS4 (Hairer and Wanner, Sec. VI.4), as the oracle derives its k-form from the published
    transformed coefficients: all eight order-4 conditions, an order-3 embedded solution that is not of
    order 4, the published nodes alpha_i and gamma_i, stiff accuracy of both solutions, and R(-inf) = 0."""
    t = small[1].tableau(method=2)
    s, g = t["s"], t["gamma"]
    assert s == 6 and g == 0.25 and t["err_order"] == 4
    a, gm, b, bh = t["alpha"][:s, :s], t["gam"][:s, :s], t["b"][:s], t["bhat"][:s]
    assert np.max(np.abs(_rosenbrock_conditions(b, a, gm, g, 4))) < 1e-14
    assert np.max(np.abs(_rosenbrock_conditions(bh, a, gm, g, 3))) < 1e-14
    assert np.min(np.abs(_rosenbrock_conditions(bh, a, gm, g, 4)[4:])) > 1e-3     # embedded: exactly order 3
    assert np.allclose(a.sum(axis=1), [0.0, 0.386, 0.21, 0.63, 1.0, 1.0], atol=1e-15)
    assert np.allclose(gm.sum(axis=1) + g, [0.25, -0.1043, 0.1035, -0.0362, 0.0, 0.0], atol=1e-14)
    # stiffly accurate: y_new is stage 6's point plus k-combination with b = last row of beta and weight gamma;
    # the embedded solution is stage 6's point itself
    beta_m = a + gm
    assert np.allclose(beta_m[s - 1, : s - 1], b[: s - 1], atol=1e-14) and abs(b[s - 1] - g) < 1e-15
    assert np.allclose(a[s - 1, : s - 1], bh[: s - 1], atol=1e-14) and bh[s - 1] == 0.0
    B = beta_m + g * np.eye(s)

    def R(z, w=b):
        return 1 + z * w @ np.linalg.solve(np.eye(s) - z * B, np.ones(s))

    assert abs(1 - b @ np.linalg.solve(B, np.ones(s))) < 1e-13 and abs(1 - bh @ np.linalg.solve(B, np.ones(s))) < 1e-13
    assert abs(R(-1e12)) < 1e-10
    assert max(abs(R(1j * y)) for y in np.logspace(-3, 6, 200)) <= 1 + 1e-12
    assert max(abs(R(x)) for x in -np.logspace(-3, 8, 200)) <= 1 + 1e-12
    # the same residual function on RODAS3 (order 3): its fourth-order conditions do not all hold
    t3 = small[1].tableau()
    r3 = _rosenbrock_conditions(t3["b"][:4], t3["alpha"][:4, :4], t3["gam"][:4, :4], t3["gamma"], 4)
    assert np.max(np.abs(r3[:4])) < 1e-15 and np.max(np.abs(r3[4:])) > 1e-3


# ------------------------------------------------------------------------------------ thermo
def test_thermo_constant_cp_special_case():
    """A NASA-7 set with only a1, a6, a7 reduces to cp/R = a1, h/RT = a1 + a6/T, s/R = a1 ln T + a7."""
    th = tm.const_cp_thermo(3.5, dhf_RT0=-10.0, s0=25.0)
    m = tm.build([0.028, 0.028], [(th, th), (th, th)], [dict(re=[(0, 1)], pr=[(1, 1)], A=1.0, rev=0)])
    o = Oracle(m)
    for T in (300.0, 999.0, 1000.0, 2500.0):
        cp, h, s = o.thermo(T)
        assert np.allclose(cp, 3.5, rtol=1e-15)
        assert np.allclose(h, 3.5 + th[5] / T, rtol=1e-14)
        assert np.allclose(s, 3.5 * math.log(T) + th[6], rtol=1e-14)


def test_thermo_derivative_identities(mid):
    """dH/dT = cp and dS/dT = cp/T for every species, both NASA ranges (central differences)."""
    m, o = mid
    rng = np.random.default_rng(0)
    for T in list(rng.uniform(320, 980, 4)) + list(rng.uniform(1020, 3000, 4)):
        d = 1e-3
        cp, _, _ = o.thermo(T)
        _, hp, sp = o.thermo(T + d)
        _, hm, sm = o.thermo(T - d)
        dH = ((T + d) * hp - (T - d) * hm) / (2 * d)      # d(H/R)/dT
        dS = (sp - sm) / (2 * d)
        assert np.allclose(dH, cp, rtol=1e-7, atol=1e-7)
        assert np.allclose(dS * T, cp, rtol=1e-7, atol=1e-7)


def test_thermo_continuity_at_tmid(mid):
    """The generator joins the two ranges at T_mid: the low set just below must match the high set at T_mid."""
    m, o = mid
    Tm = 1000.0
    below = o.thermo(Tm * (1 - 1e-13))
    at = o.thermo(Tm)
    for a, b in zip(below, at):
        assert np.allclose(a, b, rtol=1e-9, atol=1e-9)


# ------------------------------------------------------------------------------------ rate constants
def _one_reaction(rx, W=(0.02, 0.02, 0.04), cp=(3.5, 3.5, 5.0)):
    ths = [(tm.const_cp_thermo(c), tm.const_cp_thermo(c)) for c in cp]
    return tm.build(list(W), ths, [rx])


def test_arrhenius_special_cases():
    """k = A at b = 0, Ea = 0; ln k is linear in 1/T with slope -Ea/R (b = 0) and in ln T with slope b (Ea = 0)."""
    Y = np.array([0.5, 0.3, 0.2])
    o = Oracle(_one_reaction(dict(re=[(0, 1)], pr=[(1, 1)], A=3.7e5, rev=0)))
    for T in (400.0, 1500.0):
        assert o.rhs(T, P0, Y)["kf"][0] == pytest.approx(3.7e5, rel=1e-15)
    Ea = 1.234e5
    o = Oracle(_one_reaction(dict(re=[(0, 1)], pr=[(1, 1)], A=1e10, Ea=Ea, rev=0)))
    Ts = np.array([800.0, 1200.0, 2000.0])
    lk = np.log([o.rhs(T, P0, Y)["kf"][0] for T in Ts])
    slope = np.polyfit(1.0 / Ts, lk, 1)
    assert slope[0] == pytest.approx(-Ea / RU, rel=1e-12)
    assert np.max(np.abs(np.polyval(slope, 1.0 / Ts) - lk)) < 1e-11
    o = Oracle(_one_reaction(dict(re=[(0, 1)], pr=[(1, 1)], A=2.0, b=1.7, rev=0)))
    lk = np.log([o.rhs(T, P0, Y)["kf"][0] for T in Ts])
    slope = np.polyfit(np.log(Ts), lk, 1)
    assert slope[0] == pytest.approx(1.7, rel=1e-12)


def test_third_body_is_total_concentration():
    """With default efficiencies [M] = sum C = p/(Ru T) (ideal gas); a listed efficiency a adds (a-1) C_j."""
    Y = np.array([0.5, 0.3, 0.2])
    W = np.array([0.02, 0.02, 0.04])
    for eff in ({}, {2: 4.0}):
        o = Oracle(_one_reaction(dict(re=[(0, 1)], pr=[(1, 1)], A=10.0, type=1, rev=0, eff=eff)))
        for T, p in ((500.0, P0), (1800.0, 7 * P0)):
            r = o.rhs(T, p, Y)
            Wbar = 1.0 / np.sum(Y / W)
            C = p * Wbar / (RU * T) * Y / W
            M = p / (RU * T) + sum((a - 1.0) * C[j] for j, a in eff.items())
            assert r["qf"][0] / (r["kf"][0] * C[0]) == pytest.approx(M, rel=1e-13)


def _troe_rxn(alpha, T3, T1, T2=0.0, A0=5e3, Ainf=1.0):
    return dict(re=[(0, 1), (1, 1)], pr=[(2, 1)], A=Ainf, type=2, rev=0, troe=[alpha, T3, T1, T2], low=[A0, 0.0, 0.0])


def _p_for_Pr(Pr, T, A0, Ainf):
    # Pr = k0 [M] / k_inf with [M] = p / (Ru T) (all efficiencies 1, b = Ea = 0)
    return Pr * Ainf / A0 * RU * T


def test_troe_lindemann_special_case():
    """F_cent = 1 (alpha = 0, T3 -> inf, no T2) gives the Lindemann form k = k_inf Pr/(1 + Pr) exactly,
    with the limits k -> k_inf (Pr >> 1) and k -> k0 [M] (Pr << 1)."""
    o = Oracle(_one_reaction(_troe_rxn(0.0, 1e300, 1.0)))
    Y = np.array([0.4, 0.4, 0.2])
    T = 1300.0
    for Pr in (1e-6, 0.3, 1.0, 17.0, 1e6):
        k = o.rhs(T, _p_for_Pr(Pr, T, 5e3, 1.0), Y)["kf"][0]
        assert k == pytest.approx(1.0 * Pr / (1 + Pr), rel=1e-13)
    assert o.rhs(T, _p_for_Pr(1e9, T, 5e3, 1.0), Y)["kf"][0] == pytest.approx(1.0, rel=1e-8)
    k_low = o.rhs(T, _p_for_Pr(1e-9, T, 5e3, 1.0), Y)["kf"][0]
    assert k_low == pytest.approx(5e3 * _p_for_Pr(1e-9, T, 5e3, 1.0) / (RU * T), rel=1e-8)


def test_troe_broadening_landmarks():
    """The Troe broadening factor equals F_cent at the centre of the fall-off curve (log10 Pr = -c) and
    sqrt(F_cent) where the broadening variable equals +-1.  F_cent = 1/4 is set by alpha = 1/2 and
    T3 = T1 = T / ln 4."""
    T = 1250.0
    Tx = T / math.log(4.0)
    o = Oracle(_one_reaction(_troe_rxn(0.5, Tx, Tx)))
    Y = np.array([0.4, 0.4, 0.2])
    Fc = 0.25
    Lc = math.log10(Fc)
    c = -0.4 - 0.67 * Lc
    n = 0.75 - 1.27 * Lc
    for x, F in ((0.0, Fc), (n / 1.14, math.sqrt(Fc)), (-n / 0.86, math.sqrt(Fc))):
        Pr = 10.0 ** (x - c)
        k = o.rhs(T, _p_for_Pr(Pr, T, 5e3, 1.0), Y)["kf"][0]
        assert k / (Pr / (1 + Pr)) == pytest.approx(F, rel=1e-12)


# ------------------------------------------------------------------------------------ conservation
def test_mass_and_element_conservation_of_rates(mid):
    """sum_k W_k w_k = 0 and sum_k a_ek w_k = 0 (element-balanced reactions), relative to gross rates."""
    m, o = mid
    F = synth.field_bimodal_jet(m, 8, 8)
    for c in range(0, 64, 7):
        r = o.rhs(F.T[c], F.p[c], F.Y[:, c], want_gross=True)
        w = r["wdot"]
        gross_w = np.abs(r["qf"]) + np.abs(r["qr"])
        scale = np.sum(gross_w) * np.max(m.W) + 1e-300
        assert abs(np.sum(m.W * w)) <= 1e-13 * scale
        for e in range(m.comp.shape[1]):
            assert abs(np.sum(m.comp[:, e] * w)) <= 1e-13 * np.sum(gross_w) * np.max(m.comp)
        # species rates only through the stoichiometry: inert bath gas has zero net rate
        assert w[m.roles["N2"]] == 0.0


# ------------------------------------------------------------------------------------ Jacobian
def _states(m, n, seed):
    F = synth.field_uniform_random(m, n, seed=seed, T_range=(350.0, 2800.0))
    out = [(F.T[c], F.p[c], F.Y[:, c]) for c in range(n)]
    Y = F.Y[:, 0].copy()
    Y[: m.n_species // 2] = 0.0
    Y /= Y.sum()
    out.append((1500.0, 3 * P0, Y))                   # half of the species absent
    out.append((999.9, P0, F.Y[:, 1]))                # just below T_mid
    out.append((1000.0, P0, F.Y[:, 2]))               # at T_mid (high range)
    return out


@pytest.mark.parametrize("which", ["small", "mid", "large"])
def test_jacobian_matches_complex_step(which, small, mid):
    """Analytical dense Jacobian vs the complex-step derivative of the right-hand side (exact to roundoff)."""
    if which == "small":
        m, o = small
    elif which == "mid":
        m, o = mid
    else:
        m = synth.mechanism_large()
        o = Oracle(m)
    for T, p, Y in _states(m, 3 if which == "large" else 6, seed=11):
        J, G = o.jacobian(T, p, Y, want_gross=True)
        Jc = o.jacobian_cs(T, p, Y)
        assert np.all(np.abs(J - Jc) <= 1e-13 * (np.abs(Jc) + G) + 1e-300)


def test_parameter_derivative_single_reaction():
    """For a single reaction f = q e(y), so d f / d lnA = f and d f / d Ea = -f / (Ru T)."""
    rx = dict(re=[(0, 1), (1, 1)], pr=[(2, 1)], A=3e4, b=0.5, Ea=5e4, rev=1)
    o = Oracle(_one_reaction(rx, cp=(3.5, 3.5, 4.5)))
    Y = np.array([0.3, 0.3, 0.4])
    T = 1400.0
    f = o.rhs(T, P0, Y)["f"]
    assert np.allclose(o.rhs_param_cs(T, P0, Y, 0, 0), f, rtol=1e-13, atol=0)
    assert np.allclose(o.rhs_param_cs(T, P0, Y, 1, 0), -f / (RU * T), rtol=1e-13, atol=0)


# ------------------------------------------------------------------------------------ integrator
def _AB_mech(k, rev):
    th = tm.const_cp_thermo(3.5, dhf_RT0=0.0, s0=20.0)
    return tm.build([0.03, 0.03], [(th, th), (th, th)], [dict(re=[(0, 1)], pr=[(1, 1)], A=k, rev=rev)])


def test_first_order_decay_closed_form():
    """A -> B with equal W and thermo (isothermal): Y_A(t) = Y_A0 exp(-k t)."""
    k, dt = 3.0e5, 1e-5
    o = Oracle(_AB_mech(k, rev=0))
    out = o.integrate(1200.0, P0, np.array([0.9, 0.1]), dt, rtol=1e-9, atol=1e-15)
    assert out["status"] == 0
    assert out["Y"][0] == pytest.approx(0.9 * math.exp(-k * dt), rel=2e-8)
    assert out["T"] == pytest.approx(1200.0, rel=1e-14)
    assert out["Y"].sum() == pytest.approx(1.0, abs=1e-15)


def test_reversible_relaxation_closed_form():
    """A <=> B with identical thermo (Kc = 1): Y_A(t) = 1/2 + (Y_A0 - 1/2) exp(-2 k t)."""
    k, dt = 2.0e5, 1e-5
    o = Oracle(_AB_mech(k, rev=1))
    out = o.integrate(900.0, P0, np.array([0.95, 0.05]), dt, rtol=1e-9, atol=1e-15)
    assert out["Y"][0] == pytest.approx(0.5 + 0.45 * math.exp(-2 * k * dt), rel=2e-8)


def test_observed_order_three():
    """Fixed steps on A -> B: the global error falls as h^3 (order of RODAS3)."""
    k, dt = 1.0, 1.0
    o = Oracle(_AB_mech(k, rev=0))
    y0 = np.array([1000.0, 1.0, 0.0])
    errs = []
    for N in (8, 16, 32, 64):
        y = o.replay(y0, P0, np.full(N, dt / N))
        errs.append(abs(y[1] - math.exp(-k * dt)))
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(np.abs(orders - 3.0) < 0.15), orders


def test_ros2_observed_order_two_and_decay():
    """Fixed ROS2 steps on A -> B: the global error falls as h^2; the adaptive run meets the closed form."""
    k, dt = 1.0, 1.0
    o = Oracle(_AB_mech(k, rev=0))
    y0 = np.array([1000.0, 1.0, 0.0])
    errs = []
    for N in (32, 64, 128, 256):
        y = o.replay(y0, P0, np.full(N, dt / N), method=1)
        errs.append(abs(y[1] - math.exp(-k * dt)))
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(np.abs(orders - 2.0) < 0.1), orders
    r = o.integrate(1000.0, P0, np.array([1.0, 0.0]), 1.0, rtol=1e-6, atol=1e-12, method=1)
    assert r["status"] == 0 and abs(r["Y"][0] - math.exp(-1.0)) < 2e-5
    r3 = o.integrate(1000.0, P0, np.array([1.0, 0.0]), 1.0, rtol=1e-6, atol=1e-12)
    assert r["nsub"] > r3["nsub"]      # the second-order method needs more steps at the same tolerance


def test_rodas4_observed_order_four_and_decay():
    """Fixed RODAS4 steps on A -> B: the global error falls as h^4; the adaptive run meets the closed form
    with fewer steps than RODAS3 at the same tolerance."""
    k, dt = 1.0, 1.0
    o = Oracle(_AB_mech(k, rev=0))
    y0 = np.array([1000.0, 1.0, 0.0])
    errs = []
    for N in (8, 16, 32, 64):
        y = o.replay(y0, P0, np.full(N, dt / N), method=2)
        errs.append(abs(y[1] - math.exp(-k * dt)))
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(np.abs(orders - 4.0) < 0.05), orders
    r = o.integrate(1000.0, P0, np.array([1.0, 0.0]), 1.0, rtol=1e-6, atol=1e-12, method=2)
    assert r["status"] == 0 and abs(r["Y"][0] - math.exp(-1.0)) < 1e-6
    r3 = o.integrate(1000.0, P0, np.array([1.0, 0.0]), 1.0, rtol=1e-6, atol=1e-12)
    assert r["nsub"] < r3["nsub"]


def test_rodas4_self_convergence_nonlinear(small):
    """On the stiff small mechanism fixed RODAS4 steps converge at order about 4 once h is small
    (coarser steps show the order reduction of Rosenbrock methods on stiff problems)."""
    m, o = small
    F = synth.field_uniform_random(m, 4, seed=5)
    y0 = o.state(F.T[1], F.Y[:, 1])
    t_end = 2e-9
    ref = o.replay(y0, P0, np.full(4096, t_end / 4096), method=2)
    errs = []
    for N in (32, 64, 128):
        y = o.replay(y0, P0, np.full(N, t_end / N), method=2)
        errs.append(np.max(np.abs(y - ref) / (np.abs(ref) + 1e-6)))
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(orders > 3.8), orders


def test_self_convergence_order_nonlinear(small):
    """On the (nonlinear, stiff) small mechanism the fixed-step solution converges at order ~3."""
    m, o = small
    F = synth.field_uniform_random(m, 4, seed=5)
    c = 1
    y0 = o.state(F.T[c], F.Y[:, c])
    t_end = 2e-9
    ref = o.replay(y0, P0, np.full(2048, t_end / 2048))
    errs = []
    for N in (32, 64, 128):
        y = o.replay(y0, P0, np.full(N, t_end / N))
        errs.append(np.max(np.abs(y - ref) / (np.abs(ref) + 1e-6)))
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(orders > 2.6), orders


@pytest.mark.parametrize("method,rtol,atol,bar", [(0, 1e-8, 1e-16, 1e-6), (1, 1e-6, 1e-14, 5e-5),
                                                    (2, 1e-8, 1e-16, 1e-7)])
def test_agrees_with_scipy_radau(small, method, rtol, atol, bar):
    """Free-run oracle vs scipy's Radau IIA at rtol 1e-12 on the same right-hand side: RODAS3 and RODAS4
    at rtol 1e-8 (measured 3e-8 and 7e-9 at worst), ROS2 at rtol 1e-6 (a second-order method needs
    over 1e5 steps for 1e-8 on these cells; measured 8e-6), and ROS2's global error shrinking in
    proportion to its tolerance."""
    scipy_integrate = pytest.importorskip("scipy.integrate")
    m, o = small
    F = synth.field_uniform_random(m, 6, seed=7)
    for c in range(3):
        y0 = o.state(F.T[c], F.Y[:, c])
        p = F.p[c]
        dt = 2e-6
        fun = lambda t, y: o.rhs(y[0], p, y[1:])["f"]
        jac = lambda t, y: o.jacobian(y[0], p, y[1:])
        sol = scipy_integrate.solve_ivp(fun, (0, dt), y0, method="Radau", jac=jac, rtol=1e-12, atol=1e-20)
        ref = sol.y[:, -1]
        out = o.integrate(F.T[c], p, F.Y[:, c], dt, rtol=rtol, atol=atol, method=method)
        assert out["status"] == 0
        big = np.abs(ref) > 1e-8
        err = np.max(np.abs(out["y"] - ref)[big] / np.abs(ref)[big])
        assert err < bar
        if method == 1:
            tight = o.integrate(F.T[c], p, F.Y[:, c], dt, rtol=rtol / 10, atol=atol / 10, method=method)
            assert np.max(np.abs(tight["y"] - ref)[big] / np.abs(ref)[big]) < err / 5


def test_invariants_during_integration(mid):
    """Sum of Y and element masses are linear invariants (kept to roundoff by a Rosenbrock step with the
    exact Jacobian); mixture enthalpy is conserved by adiabatic constant-pressure evolution to O(rtol)."""
    m, o = mid
    F = synth.field_bimodal_jet(m, 8, 8)
    el_mass = np.array([[m.comp[k, e] / m.W[k] for e in range(m.comp.shape[1])] for k in range(m.n_species)])
    for c in (3, 40):
        out = o.integrate(F.T[c], F.p[c], F.Y[:, c], 2e-6)
        assert out["status"] == 0
        assert abs(out["Y"].sum() - F.Y[:, c].sum()) < 1e-13
        assert np.allclose(out["Y"] @ el_mass, F.Y[:, c] @ el_mass, rtol=0, atol=1e-12 * np.abs(F.Y[:, c] @ el_mass).max())

        def hmix(T, Y):
            _, h, _ = o.thermo(T)
            return np.sum(Y * h * RU * T / m.W)

        cp_scale = np.sum(F.Y[:, c] * o.thermo(F.T[c])[0] * RU / m.W) * F.T[c]
        assert abs(hmix(out["T"], out["Y"]) - hmix(F.T[c], F.Y[:, c])) < 1e-4 * cp_scale


def test_equilibrium_limit(small):
    """After a long integration every reversible reaction is in detailed balance: sum_k nu_k mu_k / RT -> 0
    with ideal-gas chemical potentials mu_k/RT = g_k + ln(C_k Ru T / p0), and dT/dt -> 0."""
    m, o = small
    F = synth.field_uniform_random(m, 4, seed=9, T_range=(1500.0, 1800.0))
    c = 0
    out = o.integrate(F.T[c], F.p[c], F.Y[:, c], 1.0, rtol=1e-10, atol=1e-20)
    assert out["status"] == 0
    T, Y, p = out["T"], out["Y"], F.p[c]
    _, h, s = o.thermo(T)
    Wbar = 1.0 / np.sum(Y / m.W)
    C = p * Wbar / (RU * T) * Y / m.W
    checked = 0
    rr = o.rhs(T, p, Y)
    for r in range(m.n_reactions):
        re, pr = m.reaction(r)
        sp = [k for k, _ in re + pr]
        if np.any(C[sp] <= 1e-200):
            continue
        # only reactions that relax well within the elapsed time can be expected in balance
        tau = np.min(C[sp]) / max(rr["qf"][r], rr["qr"][r], 1e-300)
        if tau > 1e-3:
            continue
        mu = h - s + np.log(C * RU * T / P0)
        aff = sum(nu * mu[k] for k, nu in pr) - sum(nu * mu[k] for k, nu in re)
        assert abs(aff) < 1e-6, (r, aff)
        checked += 1
    assert checked >= 8
    f = o.rhs(T, p, Y, want_gross=True)
    assert abs(f["f"][0]) < 1e-6 * f["gross"][0]


def test_replay_reproduces_free_run(small):
    """Replaying the accepted steps of a free run gives the free run's result bit for bit."""
    m, o = small
    F = synth.field_uniform_random(m, 4, seed=3)
    c = 2
    out = o.integrate(F.T[c], F.p[c], F.Y[:, c], 1e-6, trace=True)
    hs = out["trace_h"][out["trace_acc"] == 1]
    y = o.replay(o.state(F.T[c], F.Y[:, c]), F.p[c], hs)
    assert np.array_equal(y, out["y"])
    assert np.sum(hs) == pytest.approx(1e-6, rel=1e-13)


def test_discrete_sensitivities_complex_step_vs_fd(small):
    """d y_final / d (lnA_j, Ea_j, y0_i) of the replayed discrete map: complex step vs central differences."""
    m, o = small
    F = synth.field_uniform_random(m, 4, seed=4)
    c = 0
    y0 = o.state(F.T[c], F.Y[:, c])
    p = F.p[c]
    out = o.integrate(F.T[c], p, F.Y[:, c], 3e-7, trace=True)
    hs = out["trace_h"][out["trace_acc"] == 1]
    r = o.rhs(F.T[c], p, F.Y[:, c])
    top = np.argsort(-(np.abs(r["qf"]) + np.abs(r["qr"])))
    for kind, j, hfd in ((0, int(top[0]), 1e-6), (0, int(top[3]), 1e-6), (1, int(top[1]), 1.0), (2, 0, 1e-3),
                         (2, 4, 1e-9)):
        cs = o.replay_sens_cs(y0, p, hs, kind, j)
        if kind == 2:
            yp, ym = y0.copy(), y0.copy()
            yp[j] += hfd; ym[j] -= hfd
            fd = (o.replay(yp, p, hs) - o.replay(ym, p, hs)) / (2 * hfd)
        else:
            def shifted(delta):
                mm = synth.MechDesc.from_json(m.to_json())
                if kind == 0:
                    mm.A[j] *= math.exp(delta)
                    mm.low[j, 0] *= math.exp(delta)
                else:
                    mm.Ea[j] += delta
                    mm.low[j, 2] += delta
                return Oracle(mm).replay(y0, p, hs)
            fd = (shifted(hfd) - shifted(-hfd)) / (2 * hfd)
        # central differences: truncation O(h^2) plus round-off ~ eps |y| / h per component
        noise = 50 * np.finfo(float).eps * np.abs(out["y"]) / hfd
        assert np.all(np.abs(cs - fd) <= 1e-5 * np.abs(cs) + noise), (kind, j)
        assert np.abs(cs).max() > 0
