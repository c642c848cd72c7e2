"""Seeded synthetic inputs: reaction mechanisms and PaSR-like reactor states.

This module generates *inputs* only.  It holds none of the integrator's
arithmetic (no thermodynamics evaluation, no rates, no Radau step): it draws
random numbers, balances elements with integer arithmetic and converts units.
Both the FP64 CPU oracle and the CUDA path consume what it returns.

The paper integrates states drawn from partially-stirred-reactor databases of
the Burke H2 model (13 species, 27 reactions) and GRI-Mech 3.0 (53 species,
325 reactions) (Sec. 2.2, Table "PaSR parameters").  Neither the models nor
the databases are available, so both are replaced by seeded synthetic
stand-ins with the same sizes, reaction types and composition structure:

* species are element compositions over H/O/N (H2-like) or C/H/O/N
  (CH4-like); the last species is an inert bath gas (N2) that takes part in
  no reaction except as a collider;
* every reaction is element balanced and reversible; reverse rates follow
  from the NASA-7 thermo of the species (the integrator computes them);
* NASA-7 thermo: cp/R is a smooth monotone function in [2.5, 6] over
  200-3500 K; formation enthalpies follow a degree-of-reduction heuristic so
  that fuel + air -> CO2/H2O/N2 releases a realistic amount of heat;
* states mix stoichiometric fuel/air with complete-combustion products plus
  log-uniform radical traces, at PaSR-like temperatures and pressures.

Units of the returned mechanism are SI with kmol: W in kg/kmol, Arrhenius A
in (m^3/kmol)^(order-1)/s, activation temperatures Theta = Ea/R in K.
"""
from __future__ import annotations

import dataclasses
import itertools

import numpy as np

R_KJ = 8.314462618e-3          # kJ/(mol K), used only to place Ea draws in K
ATM = 101325.0                 # Pa
ATOMIC_W = {"C": 12.011, "H": 1.008, "O": 15.999, "N": 14.007}
VALENCE = {"C": 4, "H": 1, "O": 2, "N": 3}

# reaction types (shared convention of the mechanism description)
ELEMENTARY, THIRD_BODY, TROE = 0, 1, 2

MECH_H2_SEED = 1301
MECH_CH4_SEED = 5301


@dataclasses.dataclass
class Mechanism:
    """A reaction mechanism as plain arrays (the layout of ``kin_mech_desc``).

    ns, nr           species / reaction counts; species ns-1 is the inert
    names            species labels (element formulas)
    elements         element symbols, ``comp[k, e]`` atoms of element e in k
    W                [ns] molar mass, kg/kmol
    nasa             [ns, 17] T_low, T_mid, T_high, 7 low-range, 7 high-range
    reac, prod       [nr, 3] species index per stoichiometric slot, -1 = empty
                     (a species appearing twice has coefficient 2)
    arrh             [nr, 3] A (SI), b, Theta (K) of the forward rate, or of
                     k_inf for a Troe reaction
    rtype            [nr] 0 elementary, 1 third-body, 2 Troe falloff
    eff              [nr, ns] third-body efficiencies (1 = default)
    fall             [nr, 7] k0 A (SI), k0 b, k0 Theta, Troe a, T***, T*, T**
    """

    name: str
    ns: int
    nr: int
    names: list
    elements: list
    comp: np.ndarray
    W: np.ndarray
    nasa: np.ndarray
    reac: np.ndarray
    prod: np.ndarray
    arrh: np.ndarray
    rtype: np.ndarray
    eff: np.ndarray
    fall: np.ndarray
    fuel: str = ""
    hf298: np.ndarray | None = None   # generator's target enthalpies (kJ/mol), info only

    def index(self, name: str) -> int:
        return self.names.index(name)


def _parse(formula: str, elements):
    """'CH2O' -> counts over ``elements``."""
    counts = dict.fromkeys(elements, 0)
    i = 0
    while i < len(formula):
        e = formula[i]
        i += 1
        num = ""
        while i < len(formula) and formula[i].isdigit():
            num += formula[i]
            i += 1
        counts[e] += int(num) if num else 1
    return [counts[e] for e in elements]


def _formula(c, elements):
    s = ""
    for e, n in zip(elements, c):
        if n:
            s += e + (str(n) if n > 1 else "")
    return s


H2_SPECIES = ["H2", "H", "O", "O2", "OH", "H2O", "HO2", "H2O2",
              "N", "NO", "NO2", "N2O", "N2"]
CH4_CORE = ["CH4", "O2", "H2O", "CO2", "CO", "H2", "H", "O", "OH", "HO2",
            "H2O2", "CH3", "CH2", "CH", "HCO", "CH2O", "CH3O", "CH2OH",
            "CH3OH", "C2H6", "C2H5", "C2H4", "C2H3", "C2H2", "NO", "N", "NO2",
            "N2O", "NH", "NH2", "NH3", "HCN", "CN"]


def _candidate_formulas(elements, max_counts, max_atoms):
    """All plausible C/H/O/N formulas (acyclic valence bound, connected)."""
    out = []
    ranges = [range(m + 1) for m in max_counts]
    for c in itertools.product(*ranges):
        n_atoms = sum(c)
        if n_atoms == 0 or n_atoms > max_atoms:
            continue
        cd = dict(zip(elements, c))
        heavy = n_atoms - cd["H"]
        vsum = sum(VALENCE[e] * n for e, n in cd.items())
        if heavy == 0:
            if cd["H"] > 2:
                continue
        else:
            # hydrogens cannot exceed the acyclic saturation bound
            if cd["H"] > sum(cd[e] * (VALENCE[e] - 2) for e in elements if e != "H") + 2:
                continue
        if n_atoms > 1 and vsum < 2 * (n_atoms - 1):
            continue
        out.append(c)
    return out


def _species_thermo(rng, comp, elements):
    """NASA-7 coefficients for one species from seeded draws.

    cp/R(x) = c_lo + d*(2x - x^2) + eps*x^2 (1-x)^2, x = (T-200)/3300, which is
    monotone and inside [c_lo, c_lo + d] on 200-3500 K when |eps| <= d; the
    polynomial in x is re-expressed in powers of T (NASA-7 a1..a5).  The
    integration constants place h(298) and s(298) near seeded targets (a6 =
    h/R - a1*298.15, a7 = s/R - a1*ln 298.15; the remaining terms are left in,
    so the targets are approximate, which does not matter for a synthetic
    model).  The same 7 coefficients serve both temperature ranges.
    """
    cd = dict(zip(elements, comp))
    n_atoms = sum(comp)
    vsum = sum(VALENCE[e] * n for e, n in cd.items())
    radical = (vsum % 2 == 1)
    if n_atoms == 1:
        c_lo, d = 2.5, rng.uniform(0.0, 0.15)
        eps = 0.0
    elif n_atoms == 2:
        c_lo, d = rng.uniform(3.4, 3.6), rng.uniform(0.7, 1.0)
        eps = rng.uniform(-0.8, 0.8) * d
    else:
        c_lo = min(5.0, 3.8 + 0.35 * (n_atoms - 3) + rng.uniform(0.0, 0.3))
        d = min(6.0 - c_lo, rng.uniform(1.0, 2.0))
        eps = rng.uniform(-0.8, 0.8) * d
    P = np.polynomial.Polynomial
    px = P([c_lo, 2 * d, -d]) + eps * P([0, 0, 1]) * P([1, -1]) ** 2
    pT = px(P([-200.0 / 3300.0, 1.0 / 3300.0]))
    a = np.zeros(7)
    coef = pT.coef
    a[: len(coef)] = coef[:5]
    # formation enthalpy (kJ/mol): complete-oxidation products + degree of
    # reduction + radical/atom bonus + noise
    dor = 4 * cd.get("C", 0) + cd["H"] - 2 * cd["O"]
    h_prod = -393.5 * cd.get("C", 0) - 120.9 * cd["H"]
    if n_atoms == 1:
        bonus = rng.uniform(150.0, 260.0)
    elif radical:
        bonus = rng.uniform(90.0, 200.0)
    else:
        bonus = 0.0
    hf = h_prod + 110.0 * max(dor, 0) + bonus + rng.normal(0.0, 8.0 * np.sqrt(n_atoms))
    if n_atoms > 1 and not radical and dor < 0 and cd["O"] != n_atoms:
        hf += rng.uniform(40.0, 110.0)      # peroxides / N-oxides sit above products
    s_R = (rng.uniform(13.0, 19.0) if n_atoms == 1
           else 13.5 + 3.2 * (n_atoms - 1) ** 0.8 + rng.normal(0.0, 0.8))
    a[5] = hf / R_KJ - a[0] * 298.15
    a[6] = s_R - a[0] * np.log(298.15)
    return a, hf


def _arrhenius(rng, order, a_range, b_range, theta_range, kmax_cgs):
    """Draw (A_SI, b, Theta) with k below a collision-like cap on 300-3500 K."""
    Ts = np.array([300.0, 600.0, 1000.0, 1500.0, 2000.0, 2500.0, 3000.0, 3500.0])
    for _ in range(1000):
        A = 10.0 ** rng.uniform(*a_range)
        b = rng.uniform(*b_range)
        th = rng.uniform(*theta_range)
        k = A * Ts ** b * np.exp(-th / Ts)
        if np.all(k <= kmax_cgs):
            return A * 1e-3 ** (order - 1), b, th
    raise RuntimeError("could not draw Arrhenius parameters")


def make_mechanism(kind: str = "h2", seed: int | None = None) -> Mechanism:
    """Seeded synthetic mechanism.

    kind "h2": 13 species over H/O/N, 27 reactions (5 third-body, 1 Troe).
    kind "ch4": 53 species over C/H/O/N, 325 reactions (30 third-body, 15 Troe).
    """
    if kind == "h2":
        elements = ["H", "O", "N"]
        names = list(H2_SPECIES)
        n_tb, n_troe, nr = 5, 1, 27
        seed = MECH_H2_SEED if seed is None else seed
        fuel = "H2"
    elif kind == "ch4":
        elements = ["C", "H", "O", "N"]
        seed = MECH_CH4_SEED if seed is None else seed
        n_tb, n_troe, nr = 30, 15, 325
        fuel = "CH4"
        names = None
    else:
        raise ValueError(kind)
    rng = np.random.Generator(np.random.PCG64(seed))
    if kind == "ch4":
        core = list(CH4_CORE)
        core_comp = {tuple(_parse(s, elements)) for s in core}
        pool = [c for c in _candidate_formulas(elements, [3, 8, 2, 1], 9)
                if tuple(c) not in core_comp and tuple(c) != tuple(_parse("N2", elements))
                and sum(c) >= 2]
        n_extra = 52 - len(core)
        w = np.array([1.0 / (1.0 + sum(c)) ** 1.5 for c in pool])
        pick = rng.choice(len(pool), size=n_extra, replace=False, p=w / w.sum())
        names = core + [_formula(pool[i], elements) for i in sorted(pick)] + ["N2"]
    ns = len(names)
    comp = np.array([_parse(s, elements) for s in names], dtype=np.int64)
    W = comp @ np.array([ATOMIC_W[e] for e in elements])
    nasa = np.zeros((ns, 17))
    hf = np.zeros(ns)
    for k in range(ns):
        a, hf[k] = _species_thermo(rng, comp[k], elements)
        # T_low, T_mid, T_high, then the low- and high-range sets (identical)
        nasa[k, 0:3] = (200.0, 1000.0, 3500.0)
        nasa[k, 3:10] = a
        nasa[k, 10:17] = a

    inert = ns - 1
    active = list(range(ns - 1))
    key = lambda idx: tuple(comp[list(idx)].sum(axis=0))
    # all element-balanced candidates among active species
    pairs = list(itertools.combinations_with_replacement(active, 2))
    by_comp2 = {}
    for p in pairs:
        by_comp2.setdefault(key(p), []).append(p)
    by_comp1 = {}
    for s in active:
        by_comp1.setdefault(key((s,)), []).append((s,))
    triples = list(itertools.combinations_with_replacement(active, 3))
    by_comp3 = {}
    for t in triples:
        by_comp3.setdefault(key(t), []).append(t)
    exch, assoc, split3 = [], [], []
    for kk, plist in by_comp2.items():
        for a_, b_ in itertools.combinations(plist, 2):
            if set(a_) & set(b_):
                continue
            exch.append((a_, b_))
        for one in by_comp1.get(kk, []):
            for p in plist:
                if one[0] in p:
                    continue
                assoc.append((p, one))
        for t in by_comp3.get(kk, []):
            for p in plist:
                if set(p) & set(t):
                    continue
                split3.append((p, t))

    def dh(r, p):
        return hf[list(p)].sum() - hf[list(r)].sum()

    chosen = []
    used = set()

    def add(cands, kind_):
        j = rng.integers(len(cands))
        r, p = cands[j]
        sig = (tuple(sorted(r)), tuple(sorted(p)))
        if sig in used or (sig[1], sig[0]) in used:
            return False
        used.add(sig)
        chosen.append((kind_, r, p))
        return True

    # third-body and Troe reactions are association/dissociation pairs
    while sum(1 for c in chosen if c[0] == THIRD_BODY) < n_tb:
        add(assoc, THIRD_BODY)
    while sum(1 for c in chosen if c[0] == TROE) < n_troe:
        add(assoc, TROE)
    # cover every active species, then fill with exchanges (a few 2 <-> 3)
    n_elem = nr - n_tb - n_troe
    covered = set()
    for c in chosen:
        covered |= set(c[1]) | set(c[2])
    order = list(rng.permutation(active))
    for s in order:
        if s in covered:
            continue
        cands = [c for c in exch + split3 if s in c[0] or s in c[1]]
        if not cands:
            cands = [c for c in assoc if s in c[0] or s in c[1]]
            kind_ = THIRD_BODY
        else:
            kind_ = ELEMENTARY
        if kind_ == ELEMENTARY and sum(1 for c in chosen if c[0] == ELEMENTARY) >= n_elem:
            raise RuntimeError("species coverage needs more reactions")
        while not add(cands, kind_):
            pass
        covered |= set(chosen[-1][1]) | set(chosen[-1][2])
    if not covered >= set(active):
        raise RuntimeError("species coverage failed")
    n_split = max(1, n_elem // 12) if split3 else 0
    while sum(1 for c in chosen if c[0] == ELEMENTARY) < n_elem:
        use3 = split3 and sum(1 for c in chosen if c[0] == ELEMENTARY and
                              (len(c[1]) == 3 or len(c[2]) == 3)) < n_split
        add(split3 if use3 else exch, ELEMENTARY)
    # reorder: elementary first in draw order, keep types interleaved as drawn
    chosen = [chosen[i] for i in rng.permutation(len(chosen))]

    reac = -np.ones((nr, 3), dtype=np.int64)
    prod = -np.ones((nr, 3), dtype=np.int64)
    arrh = np.zeros((nr, 3))
    rtype = np.zeros(nr, dtype=np.int64)
    eff = np.ones((nr, ns))
    fall = np.zeros((nr, 7))
    water = names.index("H2O") if "H2O" in names else -1
    for i, (kind_, r, p) in enumerate(chosen):
        # write each reaction in its exothermic direction
        if dh(r, p) > 0:
            r, p = p, r
        reac[i, : len(r)] = r
        prod[i, : len(p)] = p
        rtype[i] = kind_
        order = len(r)
        if kind_ == ELEMENTARY:
            arrh[i] = _arrhenius(rng, order, (6.0, 14.0), (-1.5, 2.0),
                                 (0.0, 200.0 / R_KJ), 1e15 if order == 2 else 1e19)
        elif kind_ == THIRD_BODY:
            arrh[i] = _arrhenius(rng, order + 1, (12.0, 18.0), (-2.0, 0.0),
                                 (0.0, 50.0 / R_KJ), 1e19 if order == 2 else 1e15)
        else:
            arrh[i] = _arrhenius(rng, order, (6.0, 14.0), (-1.5, 2.0),
                                 (0.0, 50.0 / R_KJ), 1e15)
            k0 = _arrhenius(rng, order + 1, (12.0, 18.0), (-2.0, 0.0),
                            (0.0, 50.0 / R_KJ), 1e19 if order == 2 else 1e15)
            fall[i, 0:3] = k0
            fall[i, 3] = rng.uniform(0.2, 0.8)
            fall[i, 4] = rng.uniform(50.0, 500.0)
            fall[i, 5] = rng.uniform(500.0, 5000.0)
            fall[i, 6] = rng.uniform(2000.0, 1e4)
        if kind_ != ELEMENTARY:
            m = rng.integers(2, 5)
            for s in rng.choice(active, size=m, replace=False):
                eff[i, s] = rng.uniform(0.5, 6.0)
            if water >= 0 and rng.uniform() < 0.7:
                eff[i, water] = rng.uniform(5.0, 12.0)
    return Mechanism(name=f"{kind}like_seed{seed}", ns=ns, nr=nr, names=names,
                     elements=elements, comp=comp, W=W, nasa=nasa, reac=reac,
                     prod=prod, arrh=arrh, rtype=rtype, eff=eff, fall=fall,
                     fuel=fuel, hf298=hf)


# ---------------------------------------------------------------------------
# PaSR-like states
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class States:
    """A batch of constant-pressure reactor states, SoA layout.

    Y  [ns, n] mass fractions (species-major), rows sum to 1 per state
    T  [n] temperature, K
    P  [n] pressure, Pa
    """

    Y: np.ndarray
    T: np.ndarray
    P: np.ndarray

    @property
    def n(self) -> int:
        return self.T.shape[0]

    def subset(self, idx) -> "States":
        idx = np.asarray(idx)
        return States(np.ascontiguousarray(self.Y[:, idx]),
                      np.ascontiguousarray(self.T[idx]),
                      np.ascontiguousarray(self.P[idx]))


def _mass_fractions(mech: Mechanism, moles: dict) -> np.ndarray:
    x = np.zeros(mech.ns)
    for name, m in moles.items():
        x[mech.index(name)] = m
    y = x * mech.W
    return y / y.sum()


def fuel_air_and_products(mech: Mechanism):
    """Stoichiometric (phi = 1) fuel/air and its complete-combustion products.

    Air is O2 + 3.76 N2.  H2-like: 2 H2 + O2 -> 2 H2O.  CH4-like:
    CH4 + 2 O2 -> CO2 + 2 H2O.  Mass fractions, shape [ns] each.
    """
    if mech.fuel == "H2":
        unburnt = {"H2": 2.0, "O2": 1.0, "N2": 3.76}
        burnt = {"H2O": 2.0, "N2": 3.76}
    elif mech.fuel == "CH4":
        unburnt = {"CH4": 1.0, "O2": 2.0, "N2": 7.52}
        burnt = {"CO2": 1.0, "H2O": 2.0, "N2": 7.52}
    else:
        raise ValueError(mech.fuel)
    return _mass_fractions(mech, unburnt), _mass_fractions(mech, burnt)


def _compose(mech, rng, lam):
    """Y = (1-lam) Y_unburnt + lam Y_burnt, plus log-uniform radical traces."""
    yu, yb = fuel_air_and_products(mech)
    n = lam.shape[0]
    Y = (1.0 - lam)[None, :] * yu[:, None] + lam[None, :] * yb[:, None]
    majors = {mech.fuel, "O2", "N2", "H2O", "CO2"}
    minor = [k for k in range(mech.ns - 1) if mech.names[k] not in majors]
    noise = np.zeros((mech.ns, n))
    on = rng.uniform(size=(len(minor), n)) < 0.5
    vals = 10.0 ** rng.uniform(-8.0, -3.0, size=(len(minor), n))
    noise[minor, :] = np.where(on, vals, 0.0)
    s = noise.sum(axis=0)
    Y = Y * (1.0 - s)[None, :] + noise
    # the inert closes the sum exactly (it is the largest fraction)
    Y[-1, :] = 0.0
    Y[-1, :] = 1.0 - Y[:-1, :].sum(axis=0)
    return np.ascontiguousarray(Y)


def make_states(mech: Mechanism, n: int, seed: int, *, T_range=(900.0, 2500.0),
                P_atm=(1.0, 25.0), mode: str = "correlated") -> States:
    """Seeded PaSR-like states.

    mode "correlated": T ~ U(T_range); the burnt fraction follows T
      (lam = clip((T - T_lo)/(T_hi - T_lo) + N(0, 0.15), 0, 1)), so cold
      states are mostly fresh mixture and hot ones mostly products, as in a
      stirred reactor at statistical steady state.
    mode "mixed": 20 % near-equilibrium products (T ~ U(1800, 2500),
      lam ~ U(0.9, 1)) and 80 % ignition-delay states (T ~ U(900, 1200),
      lam ~ U(0, 0.1)) in random order, which makes stiffness very uneven
      across neighbouring states.
    P ~ U(P_atm) atm in both modes.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    if mode == "correlated":
        T = rng.uniform(T_range[0], T_range[1], size=n)
        lam = np.clip((T - T_range[0]) / (T_range[1] - T_range[0])
                      + rng.normal(0.0, 0.15, size=n), 0.0, 1.0)
    elif mode == "mixed":
        hot = rng.uniform(size=n) < 0.2
        T = np.where(hot, rng.uniform(1800.0, 2500.0, size=n),
                     rng.uniform(900.0, 1200.0, size=n))
        lam = np.where(hot, rng.uniform(0.9, 1.0, size=n), rng.uniform(0.0, 0.1, size=n))
    else:
        raise ValueError(mode)
    P = rng.uniform(P_atm[0], P_atm[1], size=n) * ATM
    Y = _compose(mech, rng, lam)
    return States(Y=Y, T=np.ascontiguousarray(T), P=np.ascontiguousarray(P))


# The five workloads: (mechanism kind, n, state seed, dt values, state recipe)
WORKLOADS = {
    "h2_1024": dict(kind="h2", n=1024, seed=42, dts=(1e-6,), T_range=(900.0, 2500.0),
                    mode="correlated"),
    "h2_mixed_2p20": dict(kind="h2", n=1 << 20, seed=43, dts=(1e-6, 1e-4),
                          T_range=(900.0, 2500.0), mode="mixed"),
    "ch4_2p18": dict(kind="ch4", n=1 << 18, seed=44, dts=(1e-4,), T_range=(800.0, 2600.0),
                     mode="correlated"),
    "ch4_2p16": dict(kind="ch4", n=1 << 16, seed=45, dts=(1e-6, 1e-4),
                     T_range=(800.0, 2600.0), mode="correlated"),
    "ch4_learned_test_2p20": dict(kind="ch4", n=1 << 20, seed=46, dts=(1e-4,),
                                  T_range=(800.0, 2600.0), mode="correlated"),
    "ch4_learned_train_2p20": dict(kind="ch4", n=1 << 20, seed=47, dts=(1e-4,),
                                   T_range=(800.0, 2600.0), mode="correlated"),
}


def workload(name: str, n: int | None = None):
    """(mechanism, states, dts) of a named workload; ``n`` takes a prefix."""
    w = WORKLOADS[name]
    mech = make_mechanism(w["kind"])
    nn = w["n"] if n is None else n
    st = make_states(mech, w["n"], w["seed"], T_range=w["T_range"], mode=w["mode"])
    if nn != w["n"]:
        st = st.subset(np.arange(nn))
    return mech, st, w["dts"]
