"""Seeded synthetic inputs for the per-cell chemistry step.

This module only *constructs inputs*: mechanisms written in the ``RDEMECH 1``
text format, and cell states (p, T, Y).  It evaluates no rate, no thermo
function and no step of the integrator; both the CUDA path and the CPU oracle
read what it writes, each with its own parser.

The paper's own mechanism data (San Diego H2/air, 12 species / 24 reactions,
Section 2.1) are not available, so the mechanisms here are seeded draws with the
stoichiometry of H2/O2 elementary chemistry and random Arrhenius parameters.
Cell states follow the regions of the paper's 2D RDE set-up (Section 3.2.1):
fresh stoichiometric H2/air, post-shock front, and H2O + N2 products.

Random numbers come from a counter-based splitmix64 stream: value ``i`` of
stream ``name`` under ``seed`` is ``mix64(base(seed, name) + (i + 1) * golden)``
so every quantity is reproducible and independent of how many values were drawn
before it.
"""
from __future__ import annotations

import zlib
from dataclasses import dataclass, field

import numpy as np

# ----------------------------------------------------------------------------
# splitmix64 (Steele, Lea & Flood 2014), counter form, vectorised with numpy
# ----------------------------------------------------------------------------
_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix64(z: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def _base(seed: int, name: str) -> np.uint64:
    key = np.array([(int(seed) * 0x2545F4914F6CDD1D + zlib.crc32(name.encode())) & 0xFFFFFFFFFFFFFFFF],
                   dtype=np.uint64)
    return _mix64(key)[0]


def uniform(seed: int, name: str, n: int, offset: int = 0) -> np.ndarray:
    """n doubles in [0, 1) from stream ``name``; value i is fixed by (seed, name, offset + i)."""
    idx = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = _base(seed, name) + idx * _GOLDEN
    return (_mix64(z) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def uniform_range(seed: int, name: str, n: int, lo: float, hi: float) -> np.ndarray:
    return lo + (hi - lo) * uniform(seed, name, n)


def normal(seed: int, name: str, n: int) -> np.ndarray:
    """Standard normal draws (Box-Muller on two uniform streams)."""
    u1 = uniform(seed, name + "/u1", n)
    u2 = uniform(seed, name + "/u2", n)
    return np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * np.pi * u2)


# ----------------------------------------------------------------------------
# Mechanism description and its text form
# ----------------------------------------------------------------------------
ATOMIC_MASS = {"H": 1.00794, "O": 15.9994, "N": 14.0067, "C": 12.0107, "Ar": 39.948, "X": 10.0}


@dataclass
class Species:
    name: str
    comp: dict            # element -> count
    W: float              # g/mol
    lo: list              # 7 NASA coefficients, T < Tmid
    hi: list              # 7 NASA coefficients, T >= Tmid
    Tlow: float = 200.0
    Tmid: float = 1000.0
    Thigh: float = 6000.0


@dataclass
class Reaction:
    reac: list            # [(species, coef)]
    prod: list
    A: float              # mol-cm-s units
    b: float
    E: float              # kJ/mol
    kind: str = "ELEM"    # ELEM | THREEBODY | LINDEMANN | TROE
    reversible: bool = True
    eff: dict = field(default_factory=dict)   # species -> third-body efficiency (default 1)
    low: tuple | None = None                  # (A0, b0, E0) for falloff
    troe: tuple | None = None                 # (a, T3, T1) or (a, T3, T1, T2)


@dataclass
class Mechanism:
    elements: list
    species: list
    reactions: list

    @property
    def K(self) -> int:
        return len(self.species)

    @property
    def R(self) -> int:
        return len(self.reactions)

    def index(self, name: str) -> int:
        for i, s in enumerate(self.species):
            if s.name == name:
                return i
        raise KeyError(name)

    def W_array(self) -> np.ndarray:
        return np.array([s.W for s in self.species])

    def to_text(self) -> str:
        out = ["RDEMECH 1",
               "# A in mol-cm-s units, E in kJ/mol, W in g/mol",
               "ELEMENTS %d %s" % (len(self.elements), " ".join(self.elements)),
               "SPECIES %d" % self.K]
        for s in self.species:
            counts = " ".join(str(int(s.comp.get(e, 0))) for e in self.elements)
            out.append("SP %s %.17g %.17g %.17g %.17g %s" % (s.name, s.W, s.Tlow, s.Tmid, s.Thigh, counts))
            out.append("LO " + " ".join("%.17g" % a for a in s.lo))
            out.append("HI " + " ".join("%.17g" % a for a in s.hi))
        out.append("REACTIONS %d" % self.R)
        for r in self.reactions:
            side = lambda lst: "%d %s" % (len(lst), " ".join("%s %d" % (n, c) for n, c in lst))
            out.append("RX %s %s %s %s %.17g %.17g %.17g" % (
                r.kind, "REV" if r.reversible else "IRR", side(r.reac), side(r.prod), r.A, r.b, r.E))
            if r.eff:
                out.append("EFF %d %s" % (len(r.eff), " ".join("%s %.17g" % (n, a) for n, a in r.eff.items())))
            if r.low is not None:
                out.append("LOW %.17g %.17g %.17g" % r.low)
            if r.troe is not None:
                out.append("TROE %d %s" % (len(r.troe), " ".join("%.17g" % v for v in r.troe)))
        out.append("END")
        return "\n".join(out) + "\n"


def _W(comp: dict) -> float:
    return float(sum(ATOMIC_MASS[e] * n for e, n in comp.items()))


# ----------------------------------------------------------------------------
# The seeded 9-species / 21-reaction H2-O2-N2 mechanism
# ----------------------------------------------------------------------------
H2O2_SPECIES = [
    # name, composition, formation enthalpy kJ/mol, standard entropy J/(mol K)
    ("H2", {"H": 2}, 0.0, 130.7),
    ("O2", {"O": 2}, 0.0, 205.2),
    ("H2O", {"H": 2, "O": 1}, -241.8, 188.8),
    ("H", {"H": 1}, 218.0, 114.7),
    ("O", {"O": 1}, 249.2, 161.1),
    ("OH", {"H": 1, "O": 1}, 39.0, 183.7),
    ("HO2", {"H": 1, "O": 2}, 12.0, 229.0),
    ("H2O2", {"H": 2, "O": 2}, -136.1, 232.7),
    ("N2", {"N": 2}, 0.0, 191.6),
]

# element-balanced H2/O2 elementary steps: stoichiometry only, no rate data
H2O2_STEPS = [
    ("H + O2", "O + OH"), ("O + H2", "H + OH"), ("OH + H2", "H + H2O"),
    ("2 OH", "O + H2O"), ("H2O2", "2 OH"), ("HO2 + H", "2 OH"),
    ("HO2 + H", "H2 + O2"), ("HO2 + O", "O2 + OH"), ("HO2 + OH", "H2O + O2"),
    ("2 HO2", "H2O2 + O2"), ("H2O2 + H", "H2O + OH"), ("H2O2 + H", "HO2 + H2"),
    ("H2O2 + O", "OH + HO2"), ("H2O2 + OH", "HO2 + H2O"), ("HO2 + H", "H2O + O"),
    ("H2O2 + O", "O2 + H2O"), ("H2 + HO2", "H2O + OH"), ("H2 + O2", "2 OH"),
]
H2O2_THIRD_BODY = [("2 H", "H2"), ("H + OH", "H2O"), ("H + O2", "HO2")]

_R_J = 8.31446261815324  # only to express the tabulated formation data in NASA units
_T0 = 298.15


def _parse_side(s: str) -> list:
    out = {}
    for term in s.split("+"):
        term = term.strip()
        parts = term.split()
        if len(parts) == 2:
            c, n = int(parts[0]), parts[1]
        else:
            c, n = 1, parts[0]
        out[n] = out.get(n, 0) + c
    return list(out.items())


def _atoms(comp: dict) -> int:
    return int(sum(comp.values()))


def _base_nasa(seed: int, i: int, comp: dict, dhf_kj: float, s0: float) -> list:
    """Unperturbed NASA-7 coefficients of a smooth synthetic Cp/R curve.

    Cp/R starts near 2.5 (atoms), 3.5 (diatomics), 4.0 (triatomics), 4.5 (larger)
    and rises gently with T; a6/a7 put H(298 K) and S(298 K) near the tabulated
    formation enthalpy and entropy (to within the small a2..a5 terms).
    """
    n = _atoms(comp)
    a1 = {1: 2.5, 2: 3.5, 3: 4.0}.get(n, 4.5)
    u = uniform(seed, "nasa/shape/%d" % i, 1)[0]
    s = 0.2 if n == 1 else 0.5 + u
    a2, a3, a4, a5 = s * 6e-4, -s * 5e-8, s * 1e-12, -s * 1e-16
    a6 = dhf_kj * 1e3 / _R_J - a1 * _T0
    a7 = s0 / _R_J - a1 * np.log(_T0)
    return [a1, a2, a3, a4, a5, a6, a7]


def _perturb(seed: int, i: int, coeffs: list) -> list:
    f = uniform_range(seed, "nasa/perturb/%d" % i, 7, 0.95, 1.05)
    return [float(c * fi) for c, fi in zip(coeffs, f)]


def _draw_rate(seed: int, tag: str, j: int, logA=(9.0, 17.0), b=(-1.0, 1.0), E=(0.0, 200.0)):
    u = uniform(seed, "rate/" + tag, 3 * (j + 1))[3 * j:3 * j + 3]
    return (float(10.0 ** (logA[0] + (logA[1] - logA[0]) * u[0])),
            float(b[0] + (b[1] - b[0]) * u[1]),
            float(E[0] + (E[1] - E[0]) * u[2]))


def h2_air_mechanism(seed: int = 16105) -> Mechanism:
    """Seeded 9-species / 21-reversible-reaction H2-O2-N2 mechanism.

    18 elementary steps and 3 three-body recombinations with unit efficiencies;
    log10 A ~ U[9, 17] (mol-cm-s), b ~ U[-1, 1], Ea ~ U[0, 200] kJ/mol; NASA-7
    coefficients perturbed by a factor U[0.95, 1.05] from a smooth seeded base,
    identical in both temperature ranges.
    """
    species = []
    for i, (name, comp, dhf, s0) in enumerate(H2O2_SPECIES):
        c = _perturb(seed, i, _base_nasa(seed, i, comp, dhf, s0))
        species.append(Species(name, comp, _W(comp), list(c), list(c)))
    reactions = []
    for j, (lhs, rhs) in enumerate(H2O2_STEPS):
        A, b, E = _draw_rate(seed, "elem", j)
        reactions.append(Reaction(_parse_side(lhs), _parse_side(rhs), A, b, E))
    for j, (lhs, rhs) in enumerate(H2O2_THIRD_BODY):
        A, b, E = _draw_rate(seed, "3body", j)
        reactions.append(Reaction(_parse_side(lhs), _parse_side(rhs), A, b, E, kind="THREEBODY"))
    return Mechanism(["H", "O", "N"], species, reactions)


# ----------------------------------------------------------------------------
# The seeded 53-species / 325-reaction stress mechanism
# ----------------------------------------------------------------------------
LARGE_REQUIRED = [("H", {"H": 1}), ("O", {"O": 1}), ("OH", {"H": 1, "O": 1}), ("H2", {"H": 2}),
                  ("O2", {"O": 2}), ("H2O", {"H": 2, "O": 1}), ("N2", {"N": 2}), ("Ar", {"Ar": 1}),
                  ("HO2", {"H": 1, "O": 2}), ("H2O2", {"H": 2, "O": 2})]
_FORMATION = {"H": 218.0, "O": 249.2, "OH": 39.0, "H2": 0.0, "O2": 0.0, "H2O": -241.8, "N2": 0.0, "Ar": 0.0,
              "HO2": 12.0, "H2O2": -136.1}


def _formula(comp: dict) -> str:
    out = ""
    for e in ("C", "H", "O", "N", "Ar"):
        n = comp.get(e, 0)
        if n:
            out += e + (str(n) if n > 1 else "")
    return out


def large_mechanism(seed: int = 16105, n_species: int = 53, n_reactions: int = 325, n_threebody: int = 20,
                    n_troe: int = 10) -> Mechanism:
    """Seeded element-balanced stress mechanism over {C, H, O, N, Ar}.

    Species: the H2/O2/N2/Ar set plus distinct element vectors C0-3 H0-8 O0-3 N0-2
    (at most 8 atoms).  Reactions: 1-2 reactants drawn at random; among all 1-2
    species product sets with the same element vector (other than the
    reactants), one is drawn; duplicates are rejected.  The first reactions of
    the form A + B <=> AB (or its reverse) become three-body (unit efficiencies)
    and then Troe falloff reactions.  Rate ranges as in the 9-species mechanism,
    except that an endothermic step's activation energy is raised to its
    enthalpy of reaction plus 20 kJ/mol (a non-negative reverse barrier);
    Troe k_0 over the same ranges with a ~ U[0.3, 0.8], T*** ~ U[50, 500] K,
    T* ~ U[1000, 5000] K and T** ~ U[3000, 8000] K on every second one.
    """
    elems = ["C", "H", "O", "N", "Ar"]
    cands = []
    for c in range(4):
        for h in range(9):
            for o in range(4):
                for n in range(3):
                    tot = c + h + o + n
                    if 1 <= tot <= 8:
                        comp = {k: v for k, v in (("C", c), ("H", h), ("O", o), ("N", n)) if v}
                        cands.append(comp)
    required = [c for _, c in LARGE_REQUIRED]
    pool = [c for c in cands if c not in required and not (len(c) == 1 and "N" in c and c["N"] == 1)]
    order = np.argsort(uniform(seed, "large/species", len(pool)), kind="stable")
    chosen = required + [pool[i] for i in order[: n_species - len(required)]]
    species = []
    req_names = [n for n, _ in LARGE_REQUIRED]
    for i, comp in enumerate(chosen):
        name = req_names[i] if i < len(req_names) else _formula(comp)
        atoms = _atoms(comp)
        dhf = _FORMATION.get(name)
        if dhf is None:
            dhf = float(-300.0 + 600.0 * uniform(seed, "large/dhf/%d" % i, 1)[0])
        s0 = float((100.0 + 25.0 * atoms) * (0.9 + 0.2 * uniform(seed, "large/s0/%d" % i, 1)[0]))
        base = _base_nasa(seed, 200 + i, comp, dhf, s0)
        if atoms > 4:   # larger molecules: higher Cp/R, kept below 12 on [200, 6000] K
            base[0] = min(4.5 + 0.5 * (atoms - 4), 8.0)
        c = _perturb(seed, 200 + i, base)
        species.append(Species(name, comp, _W(comp), list(c), list(c)))
    vec = {s.name: tuple(s.comp.get(e, 0) for e in elems) for s in species}
    # formation enthalpy (kJ/mol) that each species' perturbed fit carries at 298 K (leading terms)
    hf = {s.name: _R_J * (s.lo[0] * _T0 + s.lo[5]) / 1e3 for s in species}
    names = [s.name for s in species]
    by_vec = {}
    for a in range(len(names)):
        by_vec.setdefault(vec[names[a]], []).append((names[a],))
        for b in range(a, len(names)):
            v = tuple(x + y for x, y in zip(vec[names[a]], vec[names[b]]))
            by_vec.setdefault(v, []).append((names[a], names[b]))
    reactions, seen, j = [], set(), 0
    kinds = []
    while len(reactions) < n_reactions:
        u = uniform(seed, "large/rx/%d" % j, 4)
        j += 1
        nr = 1 if u[0] < 0.3 else 2
        ra = names[int(u[1] * len(names))]
        rb = names[int(u[2] * len(names))]
        reac = (ra,) if nr == 1 else tuple(sorted((ra, rb)))
        v = tuple(sum(vec[n][e] for n in reac) for e in range(5))
        opts = [pset for pset in by_vec.get(v, []) if tuple(sorted(pset)) != reac]
        if not opts:
            continue
        prod = tuple(sorted(opts[int(u[3] * len(opts))]))
        key = (reac, prod)
        if key in seen or (prod, reac) in seen:
            continue
        seen.add(key)
        side = lambda t: [(n, t.count(n)) for n in sorted(set(t))]
        A, b, E = _draw_rate(seed, "large", len(reactions))
        # thermodynamic consistency of the synthetic set: the activation energy of an
        # endothermic step is at least its enthalpy of reaction (+20 kJ/mol), so the
        # reverse step keeps a non-negative activation energy
        dH = sum(hf[n] for n in prod) - sum(hf[n] for n in reac)
        E = max(E, dH + 20.0)
        r = Reaction(side(reac), side(prod), A, b, E)
        reactions.append(r)
    # three-body and Troe: reactions joining two species into one (or splitting one into two)
    assoc = [i for i, r in enumerate(reactions)
             if (sum(c for _, c in r.reac) == 2 and sum(c for _, c in r.prod) == 1)
             or (sum(c for _, c in r.reac) == 1 and sum(c for _, c in r.prod) == 2)]
    for k, i in enumerate(assoc[: n_threebody + n_troe]):
        r = reactions[i]
        if k < n_threebody:
            r.kind = "THREEBODY"
        else:
            r.kind = "TROE"
            u = uniform(seed, "large/troe/%d" % k, 4)
            A0, b0, E0 = _draw_rate(seed, "large/k0", k)
            r.low = (A0, b0, E0)
            tr = (0.3 + 0.5 * u[0], 50.0 + 450.0 * u[1], 1000.0 + 4000.0 * u[2])
            r.troe = tr + ((3000.0 + 5000.0 * u[3],) if k % 2 == 0 else ())
    return Mechanism(elems, species, reactions)


# ----------------------------------------------------------------------------
# Small mechanisms with known solutions (test inputs)
# ----------------------------------------------------------------------------
def _flat_nasa(a1: float, a6: float, a7: float) -> list:
    return [a1, 0.0, 0.0, 0.0, 0.0, a6, a7]


def isomer_mechanism(kind: str = "ELEM", reversible: bool = False, A: float = 2.0e6, b: float = 0.0,
                     E: float = 0.0, low=None, troe=None) -> Mechanism:
    """A <=> B with identical W and thermo: isothermal, K_c = 1, first order in A.

    For kind THREEBODY the rate is multiplied by [M]; for LINDEMANN/TROE it is
    the falloff blend of ``low`` = (A0, b0, E0) and (A, b, E).  Species X (inert,
    same W) carries the third-body concentration.
    """
    th = _flat_nasa(3.5, -1000.0, 5.0)
    sp = [Species("A", {"X": 2}, 20.0, th, th), Species("B", {"X": 2}, 20.0, th, th),
          Species("X2", {"X": 2}, 20.0, th, th)]
    r = Reaction([("A", 1)], [("B", 1)], A, b, E, kind=kind, reversible=reversible, low=low, troe=troe)
    return Mechanism(["X"], sp, [r])


def dimer_mechanism(A: float = 3.0e9, b: float = 0.0, E: float = 0.0) -> Mechanism:
    """2 A -> B with W_B = 2 W_A and thermo of B twice that of A (Delta H = 0)."""
    ta = _flat_nasa(3.0, -500.0, 4.0)
    tb = [2.0 * c for c in ta]
    sp = [Species("A", {"X": 1}, 10.0, ta, ta), Species("B", {"X": 2}, 20.0, tb, tb)]
    r = Reaction([("A", 2)], [("B", 1)], A, b, E, reversible=False)
    return Mechanism(["X"], sp, [r])


def robertson_mechanism() -> Mechanism:
    """Robertson's stiff kinetics as a mechanism of three isomers.

    With equal W and identical thermo the reactor is isothermal and, at
    p = R_u * T, holds 1 mol/m^3, so mass fractions equal concentrations.
    Rate constants 0.04 1/s, 3e7 and 1e4 m^3/(mol s) are given in mol-cm-s units.
    """
    th = _flat_nasa(3.5, -1000.0, 5.0)
    sp = [Species(n, {"X": 3}, 30.0, th, th) for n in ("A", "B", "C")]
    rx = [Reaction([("A", 1)], [("B", 1)], 0.04, 0.0, 0.0, reversible=False),
          Reaction([("B", 2)], [("B", 1), ("C", 1)], 3.0e7 * 1e6, 0.0, 0.0, reversible=False),
          Reaction([("B", 1), ("C", 1)], [("A", 1), ("C", 1)], 1.0e4 * 1e6, 0.0, 0.0, reversible=False)]
    return Mechanism(["X"], sp, rx)


def dissociation_mechanism(seed: int = 16105) -> Mechanism:
    """H2 + M <=> 2 H + M with inert N2: the 3-species equilibrium test mechanism."""
    sp = []
    for i, (name, comp, dhf, s0) in enumerate([H2O2_SPECIES[0], H2O2_SPECIES[3], H2O2_SPECIES[8]]):
        c = _perturb(seed, 100 + i, _base_nasa(seed, 100 + i, comp, dhf, s0))
        sp.append(Species(name, comp, _W(comp), list(c), list(c)))
    r = Reaction([("H2", 1)], [("H", 2)], 5.0e14, 0.0, 400.0, kind="THREEBODY")
    return Mechanism(["H", "N"], sp, [r])


def two_range_mechanism() -> Mechanism:
    """Two species whose NASA fits differ between ranges but join continuously at Tmid."""
    Tm = 1000.0
    lo = [3.0, 1.0e-3, 0.0, 0.0, 0.0, -800.0, 4.0]
    # high range: same Cp, H and S at Tmid with a different split of terms
    a2h = 4.0e-4
    a1h = lo[0] + (lo[1] - a2h) * Tm
    a6h = lo[5] + (lo[0] - a1h) * Tm + (lo[1] - a2h) / 2.0 * Tm * Tm
    a7h = lo[6] + (lo[0] - a1h) * np.log(Tm) + (lo[1] - a2h) * Tm
    hi = [a1h, a2h, 0.0, 0.0, 0.0, a6h, float(a7h)]
    sp = [Species("A", {"X": 1}, 10.0, lo, hi, Tmid=Tm), Species("B", {"X": 1}, 10.0, lo, hi, Tmid=Tm)]
    r = Reaction([("A", 1)], [("B", 1)], 1.0e3, 0.0, 0.0, reversible=True)
    return Mechanism(["X"], sp, [r])


# ----------------------------------------------------------------------------
# Cell states
# ----------------------------------------------------------------------------
def _mass_fractions(mech: Mechanism, moles: dict) -> np.ndarray:
    W = mech.W_array()
    x = np.zeros(mech.K)
    for n, v in moles.items():
        x[mech.index(n)] = v
    m = x * W
    return m / m.sum()


def fresh_composition(mech: Mechanism) -> np.ndarray:
    """Stoichiometric H2/air: 2 H2 + O2 + 3.76 N2, as mass fractions."""
    return _mass_fractions(mech, {"H2": 2.0, "O2": 1.0, "N2": 3.76})


@dataclass
class CellState:
    p: np.ndarray        # [n] Pa
    T: np.ndarray        # [n] K
    Y: np.ndarray        # [K, n] species-major mass fractions
    cls: np.ndarray      # [n] int8: 0 fresh, 1 front, 2 burnt, 3 uniform mix

    @property
    def n(self) -> int:
        return int(self.T.shape[0])


def _mix_states(mech: Mechanism, seed: int, tag: str, lam: np.ndarray) -> np.ndarray:
    """Y = (1 - lam) Y_fresh + lam Y_prod, with a per-cell seeded radical pool in Y_prod."""
    n = lam.shape[0]
    W = mech.W_array()
    yf = fresh_composition(mech)
    base = np.zeros(mech.K)
    base[mech.index("H2O")] = 2.0 * W[mech.index("H2O")]
    base[mech.index("N2")] = 3.76 * W[mech.index("N2")]
    base /= base.sum()
    prod = np.repeat(base[:, None], n, axis=1)
    pool = {"OH": 1e-3, "H": 1e-4, "O": 1e-4, "H2": 1e-3, "O2": 1e-3}
    for name, y in pool.items():
        prod[mech.index(name)] += y * uniform_range(seed, "%s/pool/%s" % (tag, name), n, 0.5, 1.5)
    prod /= prod.sum(axis=0, keepdims=True)
    return (1.0 - lam)[None, :] * yf[:, None] + lam[None, :] * prod


def uniform_cells(mech: Mechanism, n: int, seed: int = 1001,
                  T=(800.0, 3000.0), p=(0.1e6, 3.0e6), lam=(0.0, 1.0)) -> CellState:
    """Independent cells with T, p and mixing fraction lambda drawn uniformly."""
    Tv = uniform_range(seed, "T", n, *T)
    pv = uniform_range(seed, "p", n, *p)
    lv = uniform_range(seed, "lambda", n, *lam)
    Y = _mix_states(mech, seed, "mix", lv)
    return CellState(pv, Tv, Y, np.full(n, 3, dtype=np.int8))


# class ranges of the RDE-like field: fresh reactants, post-shock front, burnt products
FIELD_CLASSES = {
    0: dict(T=(300.0, 600.0), p=(0.1e6, 0.3e6), lam=(0.0, 0.05)),
    1: dict(T=(1500.0, 3500.0), p=(1.0e6, 3.0e6), lam=(0.2, 0.9)),
    2: dict(T=(1800.0, 2600.0), p=(0.1e6, 1.0e6), lam=(0.95, 1.0)),
}


def field_cells(mech: Mechanism, n: int, seed: int = 1002, fractions=(0.90, 0.05, 0.05)) -> CellState:
    """RDE-like uneven field: classes fresh/front/burnt in the given fractions, order shuffled."""
    counts = [int(round(f * n)) for f in fractions]
    counts[0] = n - sum(counts[1:])
    cls = np.concatenate([np.full(c, k, dtype=np.int8) for k, c in enumerate(counts)])
    order = np.argsort(uniform(seed, "shuffle", n), kind="stable")
    cls = cls[order]
    T = np.empty(n)
    p = np.empty(n)
    lam = np.empty(n)
    for k, rng in FIELD_CLASSES.items():
        sel = cls == k
        m = int(sel.sum())
        T[sel] = uniform_range(seed, "T/%d" % k, m, *rng["T"])
        p[sel] = uniform_range(seed, "p/%d" % k, m, *rng["p"])
        lam[sel] = uniform_range(seed, "lambda/%d" % k, m, *rng["lam"])
    Y = _mix_states(mech, seed, "mix", lam)
    return CellState(p, T, Y, cls)


def block_sizes(seed: int = 1003, nblocks: int = 64, lo: float = 1e4, hi: float = 5e5) -> np.ndarray:
    """Log-uniform AMR-like block sizes."""
    u = uniform(seed, "blocks", nblocks)
    return np.floor(np.exp(np.log(lo) + (np.log(hi) - np.log(lo)) * u)).astype(np.int64)


def subset(cells: CellState, idx: np.ndarray) -> CellState:
    return CellState(cells.p[idx].copy(), cells.T[idx].copy(), np.ascontiguousarray(cells.Y[:, idx]),
                     cells.cls[idx].copy())


def sample_indices(seed: int, n: int, m: int) -> np.ndarray:
    """m distinct indices of [0, n), sorted, reproducible."""
    if m >= n:
        return np.arange(n)
    order = np.argsort(uniform(seed, "sample", n), kind="stable")
    return np.sort(order[:m])
