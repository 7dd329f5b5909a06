"""Pins of the oracle's "gross" magnitudes, the scale of the rate and Jacobian parity tolerance.

The GPU parity tests accept |gpu - oracle| <= 1e-12 (|x| + gross).  An inflated gross would make that
bar vacuous, a deflated one would make it fail on honest cancellation, so the gross sizes the oracle
returns are recomputed here without its code:

- right-hand side: for species k, W_k sum_r |nu_kr| (|q_f,r| + |q_r,r|) / rho, and for T,
  sum_k |H_k| sum_r |nu_kr| (|q_f,r| + |q_r,r|) / (rho c_p); recomputed from the per-reaction rates of
  progress the oracle returns, the stoichiometry of the description and the mixture density and heat
  capacity written out here.  Must agree to rounding.
- Jacobian: J = sum_r [e_r (grad q_f,r - grad q_r,r)^T + q_r (grad e_r)^T] with e_r = (-dH_r/(rho c_p),
  W_k nu_kr / rho).  The honest size of the terms of an entry is
      G'_ij = sum_r |e_r,i| (|d q_f,r/d y_j| + |d q_r,r/d y_j|) + (|q_f,r| + |q_r,r|) |d e_r,i/d y_j|,
  with every gradient taken here by central differences.  The oracle's G may only be larger (it also
  counts the terms inside each gradient), so G >= G' entrywise; and no row of G may exceed 10x the row
  sum of G' (a gross inflated by orders of magnitude would pass the first check and fail this one).
"""
import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2311_14941_gb300 import synth

RU = 8.314462618


def _stoich(m):
    R, n = m.n_reactions, m.n_species
    nu = np.zeros((R, n))
    for r in range(R):
        for i in range(m.reac_ptr[r], m.reac_ptr[r + 1]):
            nu[r, m.reac_sp[i]] -= m.reac_nu[i]
        for i in range(m.prod_ptr[r], m.prod_ptr[r + 1]):
            nu[r, m.prod_sp[i]] += m.prod_nu[i]
    return nu


def _mixture(o, m, y, p):
    T, Y = y[0], y[1:]
    cpR, hRT, _ = o.thermo(T)
    Wbar = 1.0 / np.sum(Y / m.W)
    rho = p * Wbar / (RU * T)
    cp = np.sum(Y * RU * cpR / m.W)
    return rho, cp, RU * T * hRT, cpR


def _e(o, m, nu, y, p):
    """e_r of every reaction: [R, m] (column 0: temperature row, 1 + k: species rows)."""
    rho, cp, H, _ = _mixture(o, m, y, p)
    E = np.empty((nu.shape[0], m.n_species + 1))
    E[:, 0] = -(nu @ H) / (rho * cp)
    E[:, 1:] = nu * m.W[None, :] / rho
    return E


def _states(m, n_rand=6):
    F = synth.field_uniform_random(m, n_rand, seed=31, T_range=(400.0, 2600.0))
    ys = [np.concatenate([[F.T[c]], F.Y[:, c]]) for c in range(n_rand)]
    ps = list(F.p)
    H = synth.field_igniting(m, 2, seed=9)
    ys += [np.concatenate([[H.T[c]], H.Y[:, c]]) for c in range(2)]
    ps += list(H.p)
    return ys, ps


@pytest.mark.parametrize("mk", [synth.mechanism_small, synth.mechanism_methane_sized])
def test_rhs_gross_recomputed_from_rates_of_progress(mk):
    m = mk()
    o = Oracle(m)
    nu = _stoich(m)
    for y, p in zip(*_states(m)):
        r = o.rhs(y[0], p, y[1:], want_gross=True)
        rho, cp, H, _ = _mixture(o, m, y, p)
        gw = np.abs(nu).T @ (np.abs(r["qf"]) + np.abs(r["qr"]))
        want = np.concatenate([[np.sum(np.abs(H) * gw) / (rho * cp)], m.W * gw / rho])
        assert np.allclose(r["gross"], want, rtol=1e-12, atol=0.0), np.max(np.abs(r["gross"] / want - 1))
        # and the gross really bounds the value (no cancellation is hidden from it)
        assert np.all(np.abs(r["f"]) <= r["gross"] * (1 + 1e-12))


@pytest.mark.parametrize("mk", [synth.mechanism_small, synth.mechanism_methane_sized])
def test_jacobian_gross_bounds_the_terms_and_is_not_inflated(mk):
    m = mk()
    o = Oracle(m)
    nu = _stoich(m)
    mm = m.n_species + 1
    for y, p in zip(*_states(m, n_rand=3)):
        J, G = o.jacobian(y[0], p, y[1:], want_gross=True)
        r0 = o.rhs(y[0], p, y[1:])
        E = _e(o, m, nu, y, p)
        dqf = np.empty((m.n_reactions, mm))
        dqr = np.empty((m.n_reactions, mm))
        dE = np.empty((m.n_reactions, mm, mm))   # [r, i, j] = d e_r,i / d y_j
        for j in range(mm):
            hj = 1e-6 * y[0] if j == 0 else 1e-7 * max(abs(y[j]), 1e-3)
            yp, ym = y.copy(), y.copy()
            yp[j] += hj
            ym[j] -= hj
            a, b = o.rhs(yp[0], p, yp[1:]), o.rhs(ym[0], p, ym[1:])
            dqf[:, j] = (a["qf"] - b["qf"]) / (2 * hj)
            dqr[:, j] = (a["qr"] - b["qr"]) / (2 * hj)
            dE[:, :, j] = (_e(o, m, nu, yp, p) - _e(o, m, nu, ym, p)) / (2 * hj)
        gq = np.abs(r0["qf"]) + np.abs(r0["qr"])
        Gp = np.abs(E).T @ (np.abs(dqf) + np.abs(dqr)) + np.einsum("r,rij->ij", gq, np.abs(dE))
        # G counts at least the honest terms (finite-difference error allowance: 1e-5 of the entry, and
        # 1e-8 of its row's largest entry for the rounding noise of differences of structural zeros)
        slack = 1e-5 * Gp + 1e-8 * Gp.max(axis=1, keepdims=True)
        assert np.all(G >= Gp - slack), np.max((Gp - G) / (Gp.max(axis=1, keepdims=True) + 1e-300))
        # the terms bound the value
        assert np.all(np.abs(J) <= G * (1 + 1e-10) + 1e-300)
        # not inflated: every row within 10x of the honest row sum
        gs, gps = G.sum(axis=1), Gp.sum(axis=1)
        assert np.all(gs[gps == 0.0] == 0.0)    # rows without terms (an inert species): no gross either
        ratio = gs[gps > 0] / gps[gps > 0]
        assert np.all(ratio <= 10.0), ratio.max()
