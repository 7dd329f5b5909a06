"""Hand-written tiny mechanisms for closed-form checks (test helper)."""
import numpy as np

from paper_2311_14941_gb300.synth import MechDesc


def const_cp_thermo(cp_R, dhf_RT0=0.0, s0=20.0, T0=300.0):
    """NASA-7 set with constant cp/R: cp/R = a1, h/RT = a1 + a6/T, s/R = a1 ln T + a7 (same for both ranges)."""
    a = np.zeros(7)
    a[0] = cp_R
    a[5] = dhf_RT0 * T0 - cp_R * T0
    a[6] = s0 - cp_R * np.log(T0)
    return a


def build(species_W, thermo, reactions, comp=None, T_mid=1000.0):
    """reactions: list of dicts with keys re, pr (lists of (sp, nu)), A, b, Ea, type (0/1/2), rev,
    eff (dict), troe (4), low (3)."""
    n = len(species_W)
    R = len(reactions)
    lo = np.array([t[0] for t in thermo], dtype=float)
    hi = np.array([t[1] for t in thermo], dtype=float)
    rp, rs, rn, pp, ps, pn, ep, es, ea = [0], [], [], [0], [], [], [0], [], []
    A = np.zeros(R); b = np.zeros(R); Ea = np.zeros(R); typ = np.zeros(R, np.int32); rev = np.zeros(R, np.int32)
    troe = np.zeros((R, 4)); low = np.zeros((R, 3))
    for r, rx in enumerate(reactions):
        for s, nu in rx["re"]:
            rs.append(s); rn.append(nu)
        for s, nu in rx["pr"]:
            ps.append(s); pn.append(nu)
        rp.append(len(rs)); pp.append(len(ps))
        for s, a in sorted(rx.get("eff", {}).items()):
            es.append(s); ea.append(a)
        ep.append(len(es))
        A[r] = rx["A"]; b[r] = rx.get("b", 0.0); Ea[r] = rx.get("Ea", 0.0)
        typ[r] = rx.get("type", 0); rev[r] = rx.get("rev", 1)
        if "troe" in rx:
            troe[r] = rx["troe"]
        if "low" in rx:
            low[r] = rx["low"]
    i32 = lambda x: np.asarray(x, dtype=np.int32)
    if comp is None:
        comp = np.zeros((n, 1), dtype=np.int32)
    return MechDesc(name="tiny", elements=["X"], species=[f"S{i}" for i in range(n)], comp=np.asarray(comp, np.int32),
                    W=np.asarray(species_W, float), nasa_lo=lo, nasa_hi=hi, T_mid=np.full(n, T_mid),
                    inert=np.zeros(n, bool), reac_ptr=i32(rp), reac_sp=i32(rs), reac_nu=i32(rn),
                    prod_ptr=i32(pp), prod_sp=i32(ps), prod_nu=i32(pn), A=A, b=b, Ea=Ea, rtype=typ,
                    reversible=rev, eff_ptr=i32(ep), eff_sp=i32(es), eff_alpha=np.asarray(ea, float),
                    troe=troe, low=low, roles={}, core=[])
