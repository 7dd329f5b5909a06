"""Seeded synthetic inputs: reaction mechanisms and cell fields.

The paper integrates the chemistry of every cell of a RANS flame (Sandia flame D with the 59-species /
356-reaction Okafor mechanism, Sec. 2.5).  Neither the mechanism file nor the flame fields are available,
so this module draws stand-ins with the same structure:

* element-balanced reversible mechanisms built from composition-matched species sets, with exchange
  reactions ``A + B <=> C + D``, third-body decompositions ``A + M <=> B + C + M`` with listed collision
  efficiencies, and Troe fall-off recombinations ``A + B (+M) <=> C``;
* NASA-7 two-range thermo for every species;
* cell fields of (T, p, Y, dt) shaped like a RANS jet flame: a cold fuel/air core, burnt product gas,
  a mixing layer between them, igniting pockets, and LTS-like per-cell time steps.

Everything here is data construction.  The module evaluates no reaction rate, equilibrium constant,
Jacobian or integrator step: the CPU oracle and the CUDA path each do that themselves from the arrays
produced here.  The only thermodynamic expression used is the NASA-7 antiderivative at the switch
temperature, needed to make the two coefficient ranges join continuously (cp, h and s) at ``T_mid``.

Both consumers take the same flat description (:class:`MechDesc`): integer index arrays and float64
parameter arrays, species-major where a matrix is involved.
"""
from __future__ import annotations

import dataclasses
import json
import math
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

# Atomic masses, kg/mol (IUPAC conventional values).
ATOMIC_MASS = {"H": 1.008e-3, "C": 12.011e-3, "N": 14.007e-3, "O": 15.999e-3}

RXN_ELEMENTARY = 0
RXN_THREE_BODY = 1
RXN_TROE = 2

ONE_ATM = 101325.0

# Atomisation (gas-phase atom formation) enthalpies, J/mol: the bond-energy model's atom energies.
ATOM_DHF = {"H": 218.0e3, "C": 717.0e3, "N": 473.0e3, "O": 249.0e3}


@dataclasses.dataclass
class MechDesc:
    """Flat mechanism description (SI units: kg/mol, mol/m^3, s, J/mol, K).

    Reactions are written in the forward direction; all reactions generated here are reversible.
    ``A``/``b``/``Ea`` are the forward modified-Arrhenius parameters (high-pressure limit for Troe).
    ``low`` holds the Troe low-pressure-limit (A0, b0, Ea0); ``troe`` holds (alpha, T3, T1, T2) with
    ``T2 <= 0`` meaning the optional T2 term is absent.  Efficiencies list only species whose collision
    efficiency differs from the default 1.
    """

    name: str
    elements: List[str]
    species: List[str]
    comp: np.ndarray          # [n, n_el] int32 atom counts
    W: np.ndarray             # [n] kg/mol
    nasa_lo: np.ndarray       # [n, 7]
    nasa_hi: np.ndarray       # [n, 7]
    T_mid: np.ndarray         # [n]
    inert: np.ndarray         # [n] bool (bath gas, in no reaction)
    reac_ptr: np.ndarray      # [R+1] int32
    reac_sp: np.ndarray       # int32
    reac_nu: np.ndarray       # int32 (>= 1)
    prod_ptr: np.ndarray
    prod_sp: np.ndarray
    prod_nu: np.ndarray
    A: np.ndarray             # [R]
    b: np.ndarray             # [R]
    Ea: np.ndarray            # [R] J/mol
    rtype: np.ndarray         # [R] int32: 0 elementary, 1 third-body, 2 Troe
    reversible: np.ndarray    # [R] int32
    eff_ptr: np.ndarray       # [R+1] int32
    eff_sp: np.ndarray        # int32
    eff_alpha: np.ndarray     # float64
    troe: np.ndarray          # [R, 4]
    low: np.ndarray           # [R, 3]
    roles: Dict[str, int] = dataclasses.field(default_factory=dict)   # fuel, O2, N2, CO2, H2O, CO, H2
    core: List[int] = dataclasses.field(default_factory=list)         # small radical-pool species

    @property
    def n_species(self) -> int:
        return len(self.species)

    @property
    def n_reactions(self) -> int:
        return int(self.A.shape[0])

    def reaction(self, r: int):
        """(reactants, products) of reaction r as lists of (species, nu)."""
        re = [(int(self.reac_sp[i]), int(self.reac_nu[i])) for i in range(self.reac_ptr[r], self.reac_ptr[r + 1])]
        pr = [(int(self.prod_sp[i]), int(self.prod_nu[i])) for i in range(self.prod_ptr[r], self.prod_ptr[r + 1])]
        return re, pr

    def to_json(self) -> str:
        d = {}
        for f in dataclasses.fields(self):
            v = getattr(self, f.name)
            d[f.name] = v.tolist() if isinstance(v, np.ndarray) else v
        return json.dumps(d)

    @staticmethod
    def from_json(text: str) -> "MechDesc":
        d = json.loads(text)
        ints = {"comp", "reac_ptr", "reac_sp", "reac_nu", "prod_ptr", "prod_sp", "prod_nu", "rtype",
                "reversible", "eff_ptr", "eff_sp"}
        kw = {}
        for f in dataclasses.fields(MechDesc):
            v = d[f.name]
            if f.name in ints:
                v = np.asarray(v, dtype=np.int32)
            elif f.name == "inert":
                v = np.asarray(v, dtype=bool)
            elif f.name in {"W", "nasa_lo", "nasa_hi", "T_mid", "A", "b", "Ea", "eff_alpha", "troe", "low"}:
                v = np.asarray(v, dtype=np.float64)
            kw[f.name] = v
        kw["roles"] = {k: int(v) for k, v in kw["roles"].items()}
        return MechDesc(**kw)


# --------------------------------------------------------------------------------------------------
# Thermo construction
# --------------------------------------------------------------------------------------------------

def _nasa_poly_for_cp(rng, n_atoms: int) -> np.ndarray:
    """cp/R(T) coefficients a1..a5 of a monotone increasing heat capacity within [2.5, 8] on 200-3500 K."""
    if n_atoms == 1:
        c_lo, c_hi = 2.5, 2.5 + rng.uniform(0.0, 0.15)
    else:
        c_lo = min(2.5 + 0.8 * (n_atoms - 1) * rng.uniform(0.8, 1.2), 6.0)
        c_hi = min(c_lo + rng.uniform(0.6, 1.2) * (n_atoms - 1), 8.0)
    # cp/R = c_lo + (c_hi - c_lo) * (1 - (1 - T/Tc)^4) for T in [0, Tc]: monotone increasing.
    Tc = 3500.0
    d = c_hi - c_lo
    # (1 - x)^4 = 1 - 4x + 6x^2 - 4x^3 + x^4, x = T/Tc
    a = np.zeros(5)
    a[0] = c_lo
    a[1] = d * 4.0 / Tc
    a[2] = -d * 6.0 / Tc ** 2
    a[3] = d * 4.0 / Tc ** 3
    a[4] = -d * 1.0 / Tc ** 4
    return a


def _antiderivative_terms(a5: np.ndarray, T: float) -> Tuple[float, float]:
    """H/R - a6 and S/R - a7 of a NASA-7 set at T (needed only to join the two ranges)."""
    h = a5[0] * T + a5[1] * T ** 2 / 2 + a5[2] * T ** 3 / 3 + a5[3] * T ** 4 / 4 + a5[4] * T ** 5 / 5
    s = a5[0] * math.log(T) + a5[1] * T + a5[2] * T ** 2 / 2 + a5[3] * T ** 3 / 3 + a5[4] * T ** 4 / 4
    return h, s


def _make_thermo(rng, n_atoms: int, dhf: float, s298_R: float, T_mid: float = 1000.0):
    """Two NASA-7 ranges that agree in cp, h and s at T_mid.

    The low range carries the monotone cp curve; the high range adds a small perturbation that vanishes at
    T_mid (so cp is continuous there) and its a6/a7 are shifted so h and s are continuous too.
    """
    lo5 = _nasa_poly_for_cp(rng, n_atoms)
    h298, s298 = _antiderivative_terms(lo5, 298.15)
    lo = np.zeros(7)
    lo[:5] = lo5
    lo[5] = dhf / 8.314462618 - h298
    lo[6] = s298_R - s298
    # perturbation eps * (T - T_mid) * (1 + q (T - T_mid)/1000), expanded in powers of T
    eps = rng.uniform(-2e-5, 2e-5) * max(n_atoms - 1, 0.2)
    q = rng.uniform(-0.2, 0.2)
    # eps*(T - Tm) + eps*q/1000*(T - Tm)^2 = eps*q/1000*T^2 + eps*(1 - 2 q Tm/1000)*T + eps*(q Tm^2/1000 - Tm)
    dlt = np.zeros(5)
    dlt[0] = eps * (q * T_mid ** 2 / 1000.0 - T_mid)
    dlt[1] = eps * (1.0 - 2.0 * q * T_mid / 1000.0)
    dlt[2] = eps * q / 1000.0
    hi5 = lo5 + dlt
    hl, sl = _antiderivative_terms(lo5, T_mid)
    hh, sh = _antiderivative_terms(hi5, T_mid)
    hi = np.zeros(7)
    hi[:5] = hi5
    hi[5] = lo[5] + hl - hh
    hi[6] = lo[6] + sl - sh
    return lo, hi


# --------------------------------------------------------------------------------------------------
# Mechanism construction
# --------------------------------------------------------------------------------------------------

def _comp_key(c) -> Tuple[int, ...]:
    return tuple(int(x) for x in c)


def _name(elements, c) -> str:
    s = "".join(f"{e}{k if k > 1 else ''}" for e, k in zip(elements, c) if k > 0)
    return s or "X"


def _candidates(elements, bounds, max_atoms):
    out = []

    def rec(i, cur):
        if i == len(elements):
            tot = sum(cur)
            if 1 <= tot <= max_atoms:
                out.append(tuple(cur))
            return
        for k in range(bounds[elements[i]] + 1):
            rec(i + 1, cur + [k])

    rec(0, [])
    return out


def make_mechanism(seed: int, n_species: int, n_reactions: int, n_three_body: int, n_troe: int,
                   elements: Sequence[str], bounds: Dict[str, int], max_atoms: int,
                   fuel: Dict[str, int], core_frac: float = 0.12, n_colliders: int = 6,
                   name: Optional[str] = None, max_tries: int = 200, a_units: str = "cgs") -> MechDesc:
    """Draw an element-balanced reversible mechanism.

    Species are distinct atom compositions (so no reaction can have a species on both sides).  A small
    radical pool ("core": the smallest compositions) mediates most reactions, as in real combustion
    mechanisms; collision efficiencies are listed only for a few small colliders plus the bath gas, which
    keeps the Jacobian pattern sparse away from the core.  Every non-inert species takes part in at least
    one reaction.  Parameter distributions: A log-uniform 1e6..1e14 in Chemkin cm-mol-s units, converted
    to SI by (1e-6)^(order-1) (``a_units="si"`` takes the numbers as SI directly), b ~ U(-1.5, 2),
    Ea ~ U(0, 200) kJ/mol; third-body efficiencies U(0.5, 12) on 3-6 listed species; Troe
    alpha ~ U(0.1, 0.9), T3 ~ logU(10, 1000) K, T1 ~ logU(500, 5000) K, T2 ~ logU(1000, 10000) K on
    half of the fall-off reactions, A0 = A_inf * 10^U(-2, 2) m^3/mol, b0 = b_inf - U(0, 1),
    Ea0 = Ea_inf * U(0, 1).
    """
    elements = list(elements)
    n_el = len(elements)
    n_elem = n_reactions - n_three_body - n_troe
    assert n_elem >= 0
    el_idx = {e: i for i, e in enumerate(elements)}

    def vec(d):
        v = [0] * n_el
        for e, k in d.items():
            v[el_idx[e]] = k
        return tuple(v)

    required = {"N2": vec({"N": 2}), "O2": vec({"O": 2}), "fuel": vec(fuel)}
    if "C" in el_idx:
        required.update({"CO2": vec({"C": 1, "O": 2}), "CO": vec({"C": 1, "O": 1})})
    if "H" in el_idx:
        required.update({"H2O": vec({"H": 2, "O": 1}), "H2": vec({"H": 2})})
    if "H" in el_idx and "O" in el_idx:
        required.update({"H": vec({"H": 1}), "O": vec({"O": 1}), "OH": vec({"O": 1, "H": 1})})

    cand_all = _candidates(elements, bounds, max_atoms)
    req_set = set(required.values())
    for attempt in range(max_tries):
        rng = np.random.default_rng([seed, attempt])
        # grow composition families: every added species is a one-atom neighbour of one already present,
        # preferring small compositions (real mechanisms are dominated by small species)
        cand_set = set(cand_all)
        have = list(dict.fromkeys(required.values()))
        parent_of: Dict[Tuple[int, ...], Tuple[int, ...]] = {}
        while len(have) < n_species:
            base = have[int(rng.integers(len(have)))]
            if base == required["N2"]:
                continue
            nbrs, wts = [], []
            for e in range(n_el):
                for dlt in (-1, 1):
                    c = list(base)
                    c[e] += dlt
                    c = tuple(c)
                    if c in cand_set and c not in have:
                        nbrs.append(c)
                        # H and O steps dominate (they are the ones a radical-pool reaction can take)
                        wts.append((1.0 if elements[e] in ("H", "O") else 0.15) / (sum(c) ** 1.5))
            if not nbrs:
                continue
            w_ = np.array(wts)
            child = nbrs[rng.choice(len(nbrs), p=w_ / w_.sum())]
            parent_of[child] = base
            have.append(child)
        comps = have
        assert len(comps) == n_species
        # shuffle species order (keeps the index order uncorrelated with roles)
        order = rng.permutation(n_species)
        comps = [comps[i] for i in order]
        index = {c: i for i, c in enumerate(comps)}
        inert = index[required["N2"]]
        reactive = [i for i in range(n_species) if i != inert]
        sizes = np.array([sum(c) for c in comps])
        # radical pool: the small H/O/C carriers first (H, O, OH, H2, O2, H2O, CO, CO2 when present),
        # then the smallest remaining species
        pool_names = [k for k in ("H", "O", "OH", "H2", "O2", "H2O", "CO", "CO2") if k in required]
        n_core = max(4, int(round(core_frac * n_species)))
        core_l = [index[required[k]] for k in pool_names][:max(n_core, 4)]
        rank = sorted((i for i in reactive if i not in core_l and i != index[required["fuel"]]),
                      key=lambda i: (sizes[i], rng.uniform()))
        core_l += rank[: max(0, n_core - len(core_l))]
        core = set(core_l)
        # formation enthalpies (J/mol) from a bond-energy model: atoms at their atomisation enthalpies
        # minus a random bond energy per bond; reference molecules O2, N2, H2 at zero, CO2/H2O/CO bound
        role_now = {k: index[v] for k, v in required.items()}
        dhf = np.zeros(n_species)
        for i, c in enumerate(comps):
            na = int(sum(c))
            atom = sum(k * ATOM_DHF[e] for e, k in zip(elements, c))
            bonds = (na - 1) * (1.0 + rng.uniform(0.0, 0.8))
            dhf[i] = float(np.clip(atom - bonds * rng.uniform(380e3, 480e3), -400e3, 450e3))
        for k in ("O2", "N2", "H2"):
            if k in role_now:
                dhf[role_now[k]] = 0.0
        for k in ("CO2", "H2O", "CO"):
            if k in role_now:
                dhf[role_now[k]] = -rng.uniform(100e3, 400e3)

        # pair sums among reactive species
        pairs: Dict[Tuple[int, ...], List[Tuple[int, int]]] = {}
        for ia, a in enumerate(reactive):
            for b in reactive[ia:]:
                s = tuple(x + y for x, y in zip(comps[a], comps[b]))
                pairs.setdefault(s, []).append((a, b))
        exch, decomp = [], []
        for s, lst in pairs.items():
            for i in range(len(lst)):
                for j in range(i + 1, len(lst)):
                    (a, b), (c, d) = lst[i], lst[j]
                    if {a, b} & {c, d}:
                        continue
                    exch.append(((a, b), (c, d)))
            if s in index and index[s] != inert:
                for (b, c) in lst:
                    decomp.append((index[s], (b, c)))

        # family-tree neighbours: parent/child and grandparent/grandchild links of the growth above
        tree_nb: Dict[int, set] = {i: set() for i in range(n_species)}
        for ch, pa in parent_of.items():
            a, b = index[ch], index[pa]
            tree_nb[a].add(b); tree_nb[b].add(a)
        for ch, pa in parent_of.items():
            if pa in parent_of:
                a, g = index[ch], index[parent_of[pa]]
                tree_nb[a].add(g); tree_nb[g].add(a)

        def one_atom(a, b):
            return b in tree_nb[a]

        # Locality, as in real mechanisms: a species outside the radical pool reacts with pool species and
        # turns into a neighbour that differs from it by one or two atoms (H-abstraction, O-addition, ...).
        def wt_exch(rx):
            (a, b), (c, d) = rx
            outside = [x for x in (a, b, c, d) if x not in core]
            if not outside:
                return 1.0
            if len(outside) == 2:
                x, y = outside
                if ((x in (a, b)) != (y in (a, b))) and one_atom(x, y):
                    return 1.0
            return 1e-3

        def wt_dec(rx):
            a, (b, c) = rx
            outside = [x for x in (a, b, c) if x not in core]
            if not outside:
                return 1.0
            if len(outside) == 2 and a in outside:
                other = b if b in outside else c
                if one_atom(a, other):
                    return 1.0
            if outside == [a]:
                return 0.5
            return 1e-3

        if not exch or not decomp:
            continue
        # elementary reactions: 2<=>2 exchanges and 1<=>2 dissociations without a third body
        elem_pool = [("x", rx) for rx in exch] + [("d", rx) for rx in decomp]

        def parts(item):
            kind, rx = item
            if kind == "x":
                return set(rx[0]) | set(rx[1])
            return {rx[0], rx[1][0], rx[1][1]}

        def wt(item):
            kind, rx = item
            return wt_exch(rx) if kind == "x" else 0.3 * wt_dec(rx)

        fuel_i, o2_i = index[required["fuel"]], index[required["O2"]]
        chosen = {"elem": [], "tb": [], "troe": []}
        quota = {"elem": n_elem, "tb": n_three_body, "troe": n_troe}
        # initiation paths: fuel and O2 decomposition, fuel + O2 exchange (when they exist)
        for sp in (fuel_i, o2_i):
            opts = [rx for rx in decomp if rx[0] == sp and rx not in chosen["tb"]]
            if opts and len(chosen["tb"]) < n_three_body:
                chosen["tb"].append(opts[rng.integers(len(opts))])
        opts = [rx for rx in exch if set(rx[0]) == {fuel_i, o2_i} or set(rx[1]) == {fuel_i, o2_i}]
        if opts and n_elem > 0:
            chosen["elem"].append(("x", opts[rng.integers(len(opts))]))
        covered = set()
        for it in chosen["elem"]:
            covered |= parts(it)
        for k in ("tb", "troe"):
            for rx in chosen[k]:
                covered |= parts(("d", rx))
        # cover every reactive species
        ok = True
        for sp in rng.permutation(reactive):
            if sp in covered:
                continue
            e_opts = [it for it in elem_pool if sp in parts(it) and it not in chosen["elem"]]
            d_opts = [rx for rx in decomp if sp in parts(("d", rx))]
            room_e = len(chosen["elem"]) < n_elem
            room_tb = len(chosen["tb"]) < n_three_body
            room_troe = len(chosen["troe"]) < n_troe
            if e_opts and room_e and (not d_opts or not (room_tb or room_troe) or rng.uniform() < 0.7):
                w_ = np.array([wt(it) for it in e_opts])
                it = e_opts[rng.choice(len(e_opts), p=w_ / w_.sum())]
                chosen["elem"].append(it)
                covered |= parts(it)
            elif d_opts and (room_tb or room_troe):
                w_ = np.array([wt_dec(rx) for rx in d_opts])
                rx = d_opts[rng.choice(len(d_opts), p=w_ / w_.sum())]
                exo = dhf[rx[0]] - dhf[rx[1][0]] - dhf[rx[1][1]] < 0.0
                if room_troe and exo and (not room_tb or rng.uniform() < 0.5):
                    chosen["troe"].append(rx)
                elif room_tb:
                    chosen["tb"].append(rx)
                else:
                    ok = False
                    break
                covered |= parts(("d", rx))
            else:
                ok = False
                break
        if not ok:
            continue
        # fill the quotas by weight; distinct stoichiometries first, duplicates only when the pool runs out
        troe_pool = [rx for rx in decomp if dhf[rx[0]] - dhf[rx[1][0]] - dhf[rx[1][1]] < 0.0]
        for key, pool_, wfun in (("elem", elem_pool, wt), ("tb", decomp, wt_dec), ("troe", troe_pool, wt_dec)):
            need = quota[key] - len(chosen[key])
            if need <= 0:
                continue
            rest = [it for it in pool_ if it not in chosen[key]]
            w_ = np.array([wfun(it) for it in rest]) if rest else np.zeros(0)
            # distinct stoichiometries: only the local ones (weight >= 0.5) here
            rest = [it for it in rest if wfun(it) >= 0.5] or rest
            w_ = np.array([wfun(it) for it in rest]) if rest else np.zeros(0)
            take = min(need, len(rest))
            if take:
                sel = rng.choice(len(rest), size=take, replace=False, p=w_ / w_.sum())
                chosen[key] += [rest[i] for i in sel]
            need -= take
            if need > 0:
                # further channels of the local pairs before any non-local stoichiometry
                w_ = np.array([wfun(it) for it in pool_])
                w_ = np.where(w_ >= 0.5, w_, w_ * 1e-3)
                sel = rng.choice(len(pool_), size=need, replace=True, p=w_ / w_.sum())
                chosen[key] += [pool_[i] for i in sel]
        break
    else:
        raise RuntimeError("could not draw a mechanism with these settings")

    # ---- species data
    W = np.array([sum(k * ATOMIC_MASS[e] for e, k in zip(elements, c)) for c in comps])
    role = {k: index[v] for k, v in required.items()}
    names = [_name(elements, c) for c in comps]
    nasa_lo = np.zeros((n_species, 7))
    nasa_hi = np.zeros((n_species, 7))
    for i, c in enumerate(comps):
        na = int(sum(c))
        s298_R = rng.uniform(16.0, 22.0) + 2.5 * (na - 1)
        nasa_lo[i], nasa_hi[i] = _make_thermo(rng, na, dhf[i], s298_R)

    # ---- colliders: a few small species + the bath gas
    coll = [role["N2"]] + sorted(core, key=lambda i: sizes[i])[: max(0, n_colliders - 1)]

    # ---- reactions: order Troe, third-body, elementary (any order is valid; this one is the file's)
    rx_list = []   # (type, reactants[(sp,nu)], products[(sp,nu)])

    def merge(sp_list):
        d: Dict[int, int] = {}
        for s in sp_list:
            d[s] = d.get(s, 0) + 1
        return sorted(d.items())

    for (a, (b, c)) in chosen["troe"]:
        rx_list.append((RXN_TROE, merge([b, c]), merge([a])))
    for (a, (b, c)) in chosen["tb"]:
        rx_list.append((RXN_THREE_BODY, merge([a]), merge([b, c])))
    for kind, rx in chosen["elem"]:
        if kind == "x":
            (a, b), (c, d) = rx
            rx_list.append((RXN_ELEMENTARY, merge([a, b]), merge([c, d])))
        else:
            a, (b, c) = rx
            rx_list.append((RXN_ELEMENTARY, merge([a]), merge([b, c])))
    # random orientation for elementary and third-body; Troe always written as the recombination
    R = len(rx_list)
    perm = rng.permutation(R)
    rx_list = [rx_list[i] for i in perm]
    rx_list.sort(key=lambda t: {RXN_TROE: 0, RXN_THREE_BODY: 1, RXN_ELEMENTARY: 2}[t[0]])
    reac_ptr, reac_sp, reac_nu = [0], [], []
    prod_ptr, prod_sp, prod_nu = [0], [], []
    eff_ptr, eff_sp, eff_alpha = [0], [], []
    A = np.zeros(R); bb = np.zeros(R); Ea = np.zeros(R)
    rtype = np.zeros(R, dtype=np.int32)
    troe = np.zeros((R, 4)); low = np.zeros((R, 3))
    for r, (t, re, pr) in enumerate(rx_list):
        if t != RXN_TROE:
            dH = sum(nu * dhf[k] for k, nu in pr) - sum(nu * dhf[k] for k, nu in re)
            if dH > 0.0:
                re, pr = pr, re
        for s, nu in re:
            reac_sp.append(s); reac_nu.append(nu)
        for s, nu in pr:
            prod_sp.append(s); prod_nu.append(nu)
        reac_ptr.append(len(reac_sp)); prod_ptr.append(len(prod_sp))
        A[r] = 10.0 ** rng.uniform(6.0, 14.0)
        if a_units == "cgs":
            order = sum(nu for _, nu in re) + (1 if t == RXN_THREE_BODY else 0)
            A[r] *= 1e-6 ** (order - 1)
        bb[r] = rng.uniform(-1.5, 2.0)
        Ea[r] = rng.uniform(0.0, 200e3)
        rtype[r] = t
        if t in (RXN_THREE_BODY, RXN_TROE):
            k = int(rng.integers(3, 7))
            k = min(k, len(coll))
            lst = sorted(rng.choice(coll, size=k, replace=False).tolist())
            for s in lst:
                eff_sp.append(int(s)); eff_alpha.append(float(rng.uniform(0.5, 12.0)))
        eff_ptr.append(len(eff_sp))
        if t == RXN_TROE:
            troe[r, 0] = rng.uniform(0.1, 0.9)
            troe[r, 1] = 10.0 ** rng.uniform(1.0, 3.0)
            troe[r, 2] = 10.0 ** rng.uniform(math.log10(500.0), math.log10(5000.0))
            troe[r, 3] = 10.0 ** rng.uniform(3.0, 4.0) if rng.uniform() < 0.5 else 0.0
            low[r, 0] = A[r] * 10.0 ** rng.uniform(-2.0, 2.0)
            low[r, 1] = bb[r] - rng.uniform(0.0, 1.0)
            low[r, 2] = Ea[r] * rng.uniform(0.0, 1.0)
    i32 = lambda x: np.asarray(x, dtype=np.int32)
    desc = MechDesc(
        name=name or f"synthetic-{n_species}sp-{R}rxn-seed{seed}", elements=elements, species=names,
        comp=np.asarray(comps, dtype=np.int32), W=W, nasa_lo=nasa_lo, nasa_hi=nasa_hi,
        T_mid=np.full(n_species, 1000.0), inert=np.array([i == role["N2"] for i in range(n_species)]),
        reac_ptr=i32(reac_ptr), reac_sp=i32(reac_sp), reac_nu=i32(reac_nu),
        prod_ptr=i32(prod_ptr), prod_sp=i32(prod_sp), prod_nu=i32(prod_nu),
        A=A, b=bb, Ea=Ea, rtype=rtype, reversible=np.ones(R, dtype=np.int32),
        eff_ptr=i32(eff_ptr), eff_sp=i32(eff_sp), eff_alpha=np.asarray(eff_alpha, dtype=np.float64),
        troe=troe, low=low, roles=role, core=sorted(int(i) for i in core))
    check_balance(desc)
    return desc


def check_balance(m: MechDesc) -> None:
    """Raise if a reaction does not conserve every element."""
    for r in range(m.n_reactions):
        re, pr = m.reaction(r)
        lhs = sum(nu * m.comp[s] for s, nu in re)
        rhs = sum(nu * m.comp[s] for s, nu in pr)
        if not np.array_equal(lhs, rhs):
            raise ValueError(f"reaction {r} is not element balanced")


# Named workloads ----------------------------------------------------------------------------------

def mechanism_small(seed: int = 10271, a_units: str = "cgs") -> MechDesc:
    """10 species (H, O, N; one inert N2-like bath gas), 27 reversible reactions, 3 Troe, 4 third-body."""
    return make_mechanism(seed, 10, 27, 4, 3, ["H", "O", "N"], {"H": 2, "O": 3, "N": 2}, 4,
                          fuel={"H": 2}, core_frac=0.4, n_colliders=4, name="small-10sp-27rxn",
                          a_units=a_units)


def mechanism_methane_sized(seed: int = 53325, a_units: str = "cgs") -> MechDesc:
    """53 species (C, H, O, N), 325 reversible reactions: 30 third-body, 25 Troe fall-off."""
    return make_mechanism(seed, 53, 325, 30, 25, ["C", "H", "O", "N"], {"C": 2, "H": 6, "O": 3, "N": 2}, 7,
                          fuel={"C": 1, "H": 4}, core_frac=0.12, name="methane-sized-53sp-325rxn",
                          a_units=a_units)


def mechanism_large(seed: int = 1501000, a_units: str = "cgs") -> MechDesc:
    """150 species (C, H, O, N), 1000 reversible reactions: 100 third-body, 60 Troe fall-off."""
    return make_mechanism(seed, 150, 1000, 100, 60, ["C", "H", "O", "N"], {"C": 4, "H": 10, "O": 4, "N": 2}, 10,
                          fuel={"C": 1, "H": 4}, core_frac=0.04, name="large-150sp-1000rxn",
                          a_units=a_units)


# --------------------------------------------------------------------------------------------------
# Cell fields
# --------------------------------------------------------------------------------------------------

@dataclasses.dataclass
class Field:
    """Cell states, structure of arrays: ``Y[k, c]`` is species k of cell c (species-major)."""
    T: np.ndarray
    p: np.ndarray
    Y: np.ndarray
    dt: np.ndarray
    kind: np.ndarray    # per-cell label: 0 cold/unburnt, 1 burnt, 2 mixing, 3 igniting, 4 random

    @property
    def n_cells(self) -> int:
        return int(self.T.shape[0])

    def subset(self, idx) -> "Field":
        idx = np.asarray(idx)
        return Field(self.T[idx].copy(), self.p[idx].copy(), self.Y[:, idx].copy(), self.dt[idx].copy(),
                     self.kind[idx].copy())


def _moles_to_Y(m: MechDesc, X: np.ndarray) -> np.ndarray:
    """Mole numbers [n, N] -> mass fractions [n, N]."""
    mass = X * m.W[:, None]
    return mass / mass.sum(axis=0, keepdims=True)


def _fuel_air_moles(m: MechDesc, phi: np.ndarray) -> np.ndarray:
    """Mole numbers of fuel + air (O2:N2 = 21:79) at equivalence ratio phi, per cell."""
    el = {e: i for i, e in enumerate(m.elements)}
    fc = m.comp[m.roles["fuel"]]
    c = fc[el["C"]] if "C" in el else 0
    h = fc[el["H"]] if "H" in el else 0
    o = fc[el["O"]] if "O" in el else 0
    s = c + h / 4.0 - o / 2.0          # O2 per fuel for complete oxidation
    N = phi.shape[0]
    X = np.zeros((m.n_species, N))
    X[m.roles["fuel"]] = phi
    X[m.roles["O2"]] = s
    X[m.roles["N2"]] += s * 79.0 / 21.0
    return X


def _burnt_moles(m: MechDesc, phi: np.ndarray) -> np.ndarray:
    """Product-gas mole numbers for fuel/air at phi: complete oxidation when lean; CO/H2 when rich."""
    el = {e: i for i, e in enumerate(m.elements)}
    fc = m.comp[m.roles["fuel"]]
    c = fc[el["C"]] if "C" in el else 0
    h = fc[el["H"]] if "H" in el else 0
    o = fc[el["O"]] if "O" in el else 0
    s = c + h / 4.0 - o / 2.0
    N = phi.shape[0]
    X = np.zeros((m.n_species, N))
    X[m.roles["N2"]] = s * 79.0 / 21.0
    O_atoms = 2.0 * s + o * phi         # per phi units of fuel
    C_atoms = c * phi
    H_atoms = h * phi
    lean = phi <= 1.0
    if "CO2" in m.roles:
        X[m.roles["CO2"]] = np.where(lean, C_atoms, 0.0)
    if "H2O" in m.roles:
        X[m.roles["H2O"]] = np.where(lean, H_atoms / 2.0, 0.0)
    X[m.roles["O2"]] = np.where(lean, (O_atoms - 2 * C_atoms - H_atoms / 2.0) / 2.0, 0.0)
    # rich: C -> CO, then O -> H2O, leftover H -> H2 (O is sufficient for phi <= 2 with the fuels used here)
    rich = ~lean
    o_left = O_atoms - C_atoms
    if "CO" in m.roles:
        X[m.roles["CO"]] = np.where(rich, C_atoms, X[m.roles["CO"]])
    if "H2O" in m.roles:
        h2o = np.minimum(o_left, H_atoms / 2.0)
        X[m.roles["H2O"]] = np.where(rich, h2o, X[m.roles["H2O"]])
        if "H2" in m.roles:
            X[m.roles["H2"]] = np.where(rich, H_atoms / 2.0 - h2o, X[m.roles["H2"]])
    return np.maximum(X, 0.0)


def _add_radicals_and_noise(m: MechDesc, rng, X: np.ndarray, lo=-4.0, hi=-2.0, noise=0.01) -> np.ndarray:
    tot = X.sum(axis=0, keepdims=True)
    majors = {m.roles.get(k) for k in ("O2", "N2", "CO2", "H2O", "CO", "H2", "fuel")}
    for k in m.core:
        if k in majors:
            continue
        X[k] += tot[0] * 10.0 ** rng.uniform(lo, hi, size=X.shape[1])
    X = X * np.exp(noise * rng.standard_normal(X.shape))
    return X


def field_uniform_random(m: MechDesc, n_cells: int, seed: int = 1, T_range=(900.0, 2200.0),
                         dt: float = 1e-5, p: float = ONE_ATM) -> Field:
    """p = 1 atm, T ~ U(T_range), Y ~ Dirichlet(1) over all species, uniform dt."""
    rng = np.random.default_rng(seed)
    T = rng.uniform(*T_range, size=n_cells)
    Y = rng.dirichlet(np.ones(m.n_species), size=n_cells).T.copy()
    return Field(T, np.full(n_cells, p), Y, np.full(n_cells, dt), np.full(n_cells, 4, dtype=np.int32))


def field_bimodal_jet(m: MechDesc, nx: int, ny: int, seed: int = 2, dt=1e-5, dt_range=None,
                      p: float = ONE_ATM) -> Field:
    """A 2-D jet-flame-like field of nx*ny cells.

    Radial distance r from the jet axis sets a mixing variable w = 0.5 (1 + tanh((r0 - r)/delta)): about
    40 % of the cells are unburnt fuel/air (T ~ U(300, 600) K, phi ~ U(0.6, 1.6)), about 60 % are burnt
    product gas (T ~ U(1600, 2200) K, products of the local phi plus pool radicals at mole fractions
    1e-4..1e-2, 1 % log-normal noise), and the ~10 % of cells with 0.05 < w < 0.95 form a mixing layer
    in which Y and T are the w-weighted blends of the two states.  ``dt`` is uniform unless
    ``dt_range`` = (lo, hi) asks for log-uniform per-cell steps.
    """
    rng = np.random.default_rng(seed)
    N = nx * ny
    j = np.arange(N) % ny
    i = np.arange(N) // ny
    # radius from the axis with a slow axial spreading of the jet
    r = np.abs(j - (ny - 1) / 2.0) / (ny / 2.0)
    spread = 1.0 + 0.6 * i / max(nx - 1, 1)
    x = r / spread
    # r0 chosen so that ~40 % of cells have w > 0.5; delta so that ~10 % lie in the layer
    r0 = np.quantile(x, 0.40)
    delta = 0.025
    w = 0.5 * (1.0 + np.tanh((r0 - x) / delta))
    phi = rng.uniform(0.6, 1.6, size=N)
    Xu = _fuel_air_moles(m, phi)
    Xb = _add_radicals_and_noise(m, rng, _burnt_moles(m, phi))
    Yu = _moles_to_Y(m, Xu)
    Yb = _moles_to_Y(m, Xb)
    Tu = rng.uniform(300.0, 600.0, size=N)
    Tb = rng.uniform(1600.0, 2200.0, size=N)
    Y = w * Yu + (1.0 - w) * Yb
    Y /= Y.sum(axis=0, keepdims=True)
    T = w * Tu + (1.0 - w) * Tb
    kind = np.where(w > 0.95, 0, np.where(w < 0.05, 1, 2)).astype(np.int32)
    if dt_range is None:
        dts = np.full(N, dt)
    else:
        dts = 10.0 ** rng.uniform(math.log10(dt_range[0]), math.log10(dt_range[1]), size=N)
    return Field(T, np.full(N, p), Y, dts, kind)


def field_lts_mix(m: MechDesc, n_cells: int, seed: int = 3, dt_range=(1e-7, 1e-3), p: float = ONE_ATM) -> Field:
    """Heavy-tailed stiffness mix with LTS-like steps: 70 % frozen cold fuel/air (300-600 K), 20 % burnt
    (1600-2200 K), 10 % igniting fuel/air at 1000-1300 K with phi in [0.5, 0.8] U [1.3, 2.0]; per-cell dt
    log-uniform over ``dt_range``, independent of the cell kind."""
    rng = np.random.default_rng(seed)
    N = n_cells
    u = rng.uniform(size=N)
    kind = np.where(u < 0.7, 0, np.where(u < 0.9, 1, 3)).astype(np.int32)
    phi_cold = rng.uniform(0.6, 1.6, size=N)
    lean = rng.uniform(size=N) < 0.5
    phi_ign = np.where(lean, rng.uniform(0.5, 0.8, size=N), rng.uniform(1.3, 2.0, size=N))
    phi = np.where(kind == 3, phi_ign, phi_cold)
    Xu = _fuel_air_moles(m, phi)
    Xb = _add_radicals_and_noise(m, rng, _burnt_moles(m, phi))
    Y = np.where(kind[None, :] == 1, _moles_to_Y(m, Xb), _moles_to_Y(m, Xu))
    T = np.where(kind == 0, rng.uniform(300.0, 600.0, size=N),
                 np.where(kind == 1, rng.uniform(1600.0, 2200.0, size=N), rng.uniform(1000.0, 1300.0, size=N)))
    dts = 10.0 ** rng.uniform(math.log10(dt_range[0]), math.log10(dt_range[1]), size=N)
    return Field(T, np.full(N, p), Y, dts, kind)


def field_igniting(m: MechDesc, n_cells: int, seed: int = 4, dt: float = 1e-3) -> Field:
    """Igniting fuel/air cells: T0 ~ U(1000, 1400) K, p ~ logU(1, 10) atm, phi ~ U(0.6, 1.6)."""
    rng = np.random.default_rng(seed)
    N = n_cells
    phi = rng.uniform(0.6, 1.6, size=N)
    Y = _moles_to_Y(m, _fuel_air_moles(m, phi))
    T = rng.uniform(1000.0, 1400.0, size=N)
    p = ONE_ATM * 10.0 ** rng.uniform(0.0, 1.0, size=N)
    return Field(T, p, Y, np.full(N, dt), np.full(N, 3, dtype=np.int32))


def cotangent_species(m: MechDesc, n: int = 5, seed: int = 4) -> List[int]:
    """A seeded pick of ``n`` non-inert species whose final mass fractions enter the adjoint objective."""
    rng = np.random.default_rng(seed + 1000)
    cand = [k for k in range(m.n_species) if not m.inert[k]]
    return sorted(int(k) for k in rng.choice(cand, size=n, replace=False))
