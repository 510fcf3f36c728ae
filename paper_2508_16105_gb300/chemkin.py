"""Import and export of mechanisms in the CHEMKIN-II text format.

Mechanisms such as the paper's San Diego H2/air set are distributed as a
CHEMKIN-II mechanism file (ELEMENTS, SPECIES, REACTIONS) with NASA-7 polynomials
in a THERMO section or a separate thermo file.  `read_chemkin` turns them into a
`synth.Mechanism`, whose `to_text()` is the RDEMECH 1 text `rde_mech_load` takes;
`write_chemkin` writes a mechanism back in that format.

Supported: element and species lists (with optional /weight/ after an element);
THERMO sections with a global temperature line and 4-line NASA-7 records (fixed
15-character coefficient fields); reaction units (CAL/MOLE default, KCAL/MOLE,
JOULES/MOLE, KJOULES/MOLE, KELVINS; MOLES); `=`, `<=>` and `=>`; integer
stoichiometric coefficients (`2OH`, `2 OH`); third bodies `+M` with efficiencies
(`H2/2.5/`); falloff `(+M)` with LOW and optional TROE (3 or 4 parameters);
falloff with one named collider `(+AR)` (efficiency 1 for it, 0 for all others);
DUPLICATE.  Refused with a ValueError naming the line: REV, SRI, PLOG, CHEB,
HIGH, FORD / RORD, MOLECULES units, non-integer coefficients.
"""
from __future__ import annotations

import re

from .synth import Mechanism, Reaction, Species

# standard atomic weights (g/mol); H, C, N, O and Ar as in synth.ATOMIC_MASS
ATOMIC_WEIGHT = {"H": 1.00794, "D": 2.014102, "He": 4.002602, "C": 12.0107, "N": 14.0067, "O": 15.9994,
                 "F": 18.9984032, "Ne": 20.1797, "Si": 28.0855, "S": 32.065, "Cl": 35.453, "Ar": 39.948,
                 "Kr": 83.798, "Xe": 131.293, "X": 10.0}

# activation energy conversion to kJ/mol
_E_UNITS = {"CAL/MOLE": 4.184e-3, "KCAL/MOLE": 4.184, "JOULES/MOLE": 1e-3, "KJOULES/MOLE": 1.0,
            "KJ/MOLE": 1.0, "KELVINS": 8.31446261815324e-3, "EVOLTS": 96.48533212}
_UNSUPPORTED = ("REV", "SRI", "PLOG", "CHEB", "HIGH", "FORD", "RORD", "LT", "RLT", "TDEP", "EXCI", "JAN", "FIT1",
                "MOME", "XSMI", "USRPROG")


def _element_name(s: str) -> str:
    return s[:1].upper() + s[1:].lower()


def _strip_comment(line: str) -> str:
    i = line.find("!")
    return line if i < 0 else line[:i]


def _sections(text: str) -> dict:
    """Split the text into its keyword sections: name -> (header words, [(line number, line)])."""
    out, cur = {}, None
    for no, raw in enumerate(text.splitlines(), 1):
        line = _strip_comment(raw) if cur != "THERMO" else raw.rstrip("\n")
        words = line.split()
        if cur != "THERMO" and not words:
            continue
        key = words[0].upper() if words else ""
        if cur is None or (cur != "THERMO" and key in ("ELEMENTS", "ELEM", "SPECIES", "SPEC", "THERMO",
                                                      "REACTIONS", "REAC")):
            if key in ("ELEMENTS", "ELEM"):
                cur = "ELEMENTS"
            elif key in ("SPECIES", "SPEC"):
                cur = "SPECIES"
            elif key == "THERMO":
                cur = "THERMO"
            elif key in ("REACTIONS", "REAC"):
                cur = "REACTIONS"
            elif key == "END":
                continue
            else:
                raise ValueError("line %d: text outside a section: %r" % (no, raw.strip()))
            out.setdefault(cur, ([w.upper() for w in words[1:]], []))
            if cur in ("ELEMENTS", "SPECIES") and len(words) > 1:
                out[cur][1].append((no, " ".join(words[1:])))
            continue
        if cur == "THERMO":
            if line.strip().upper().startswith("END"):
                cur = None
                continue
            out[cur][1].append((no, raw))
            continue
        if key == "END":
            cur = None
            continue
        out[cur][1].append((no, line))
    return out


def _parse_elements(lines) -> tuple:
    names, weights = [], {}
    for no, line in lines:
        for m in re.finditer(r"([A-Za-z][A-Za-z0-9]*)\s*(?:/\s*([^/]+)/)?", line):
            e = _element_name(m.group(1))
            if e.upper() == "END":
                continue
            names.append(e)
            if m.group(2):
                weights[e] = float(m.group(2))
    return names, weights


def _parse_thermo(lines, wanted: set) -> dict:
    """NASA-7 records: name -> (composition, Tlow, Tmid, Thigh, lo[7], hi[7])."""
    lines = [(no, l) for no, l in lines if l.strip() and not l.lstrip().startswith("!")]
    tmid_default = 1000.0
    if lines and not lines[0][1].rstrip().endswith("1"):
        try:
            vals = [float(v) for v in lines[0][1].split()[:3]]
            if len(vals) == 3:
                tmid_default = vals[1]
                lines = lines[1:]
        except ValueError:
            pass
    out, i = {}, 0
    while i < len(lines):
        no, l1 = lines[i]
        if i + 3 >= len(lines):
            raise ValueError("line %d: incomplete NASA-7 record" % no)
        l1 = l1.ljust(80)
        name = l1[0:18].split()[0] if l1[0:18].split() else ""
        comp = {}
        for k in range(4):
            f = l1[24 + 5 * k: 29 + 5 * k]
            el, cnt = f[:2].strip(), f[2:].strip()
            if el and cnt and float(cnt) != 0.0:
                comp[_element_name(el)] = comp.get(_element_name(el), 0) + int(round(float(cnt)))
        tlow, thigh = float(l1[45:55]), float(l1[55:65])
        tmid = float(l1[65:73]) if l1[65:73].strip() else tmid_default
        coeffs = []
        for j in range(1, 4):
            lj = lines[i + j][1].ljust(80)
            for k in range(5 if j < 3 else 4):
                field = lj[15 * k: 15 * (k + 1)].strip()
                if not field:
                    raise ValueError("line %d: missing NASA-7 coefficient" % lines[i + j][0])
                coeffs.append(float(field.replace("D", "E").replace("d", "e")))
        if name in wanted and name not in out:
            out[name] = (comp, tlow, tmid, thigh, coeffs[7:14], coeffs[0:7])
        i += 4
    return out


_SPLIT = re.compile(r"<=>|=>|=")


def _side(expr: str, names: set, no: int):
    """Species and integer coefficients of one side, and its third-body marker."""
    third, falloff = None, None
    m = re.search(r"\(\+\s*([A-Za-z0-9_()*,\-]+?)\s*\)\s*$", expr)
    if m:
        falloff = m.group(1)
        expr = expr[:m.start()]
    terms = [t.strip() for t in re.split(r"\+(?![^(]*\))", expr) if t.strip()]
    out = []
    for t in terms:
        if t.upper() == "M":
            third = "M"
            continue
        t = t.replace(" ", "")
        if t in names:
            out.append((t, 1))
            continue
        m2 = re.match(r"^(\d+(?:\.\d*)?)(.+)$", t)
        if not m2 or m2.group(2) not in names:
            raise ValueError("line %d: unknown species %r" % (no, t))
        c = float(m2.group(1))
        if c != int(c):
            raise ValueError("line %d: non-integer coefficient %r" % (no, t))
        out.append((m2.group(2), int(c)))
    merged = {}
    for n, c in out:
        merged[n] = merged.get(n, 0) + c
    return list(merged.items()), third, falloff


def read_chemkin(mech_text: str, thermo_text: str | None = None) -> Mechanism:
    """Parse a CHEMKIN-II mechanism (and thermo file, when the mechanism has no THERMO
    section) into a Mechanism.  Species W comes from the element weights."""
    sec = _sections(mech_text)
    if "ELEMENTS" not in sec or "SPECIES" not in sec or "REACTIONS" not in sec:
        raise ValueError("ELEMENTS, SPECIES and REACTIONS sections are required")
    elements, ew = _parse_elements(sec["ELEMENTS"][1])
    names = []
    for no, line in sec["SPECIES"][1]:
        names.extend(w for w in line.split() if w.upper() != "END")
    if len(set(names)) != len(names):
        raise ValueError("duplicate species")
    if "THERMO" in sec:
        tlines = sec["THERMO"][1]
    elif thermo_text is not None:
        tlines = _sections("THERMO\n" + re.sub(r"(?im)^\s*THERMO.*$", "", thermo_text, count=1))["THERMO"][1]
    else:
        raise ValueError("no THERMO section and no thermo text")
    th = _parse_thermo(tlines, set(names))
    weights = dict(ATOMIC_WEIGHT)
    weights.update(ew)
    species = []
    for n in names:
        if n not in th:
            raise ValueError("no thermo data for species %s" % n)
        comp, tlow, tmid, thigh, lo, hi = th[n]
        for e in comp:
            if e not in elements:
                raise ValueError("species %s uses element %s, which ELEMENTS does not list" % (n, e))
            if e not in weights:
                raise ValueError("no atomic weight for element %s (give it as %s /weight/)" % (e, e))
        W = float(sum(weights[e] * c for e, c in comp.items()))
        species.append(Species(n, comp, W, lo, hi, tlow, tmid, thigh))
    # reactions
    units = sec["REACTIONS"][0]
    efac = _E_UNITS["CAL/MOLE"]
    for u in units:
        if u in _E_UNITS:
            efac = _E_UNITS[u]
        elif u == "MOLECULES":
            raise ValueError("REACTIONS MOLECULES units are not supported")
        elif u != "MOLES":
            raise ValueError("unknown REACTIONS unit %s" % u)
    nameset = set(names)
    reactions, cur = [], None
    for no, line in sec["REACTIONS"][1]:
        text = line.strip()
        if not text:
            continue
        if _SPLIT.search(text) and not text.upper().startswith(("LOW", "TROE")):
            parts = text.split()
            if len(parts) < 4:
                raise ValueError("line %d: reaction needs A, b and E" % no)
            try:
                A, b, E = float(parts[-3]), float(parts[-2]), float(parts[-1])
            except ValueError:
                raise ValueError("line %d: reaction needs A, b and E" % no) from None
            eq = "".join(parts[:-3])
            op = _SPLIT.search(eq).group(0)
            lhs, rhs = eq.split(op, 1)
            reac, t1, f1 = _side(lhs, nameset, no)
            prod, t2, f2 = _side(rhs, nameset, no)
            if (t1 is None) != (t2 is None) or (f1 is None) != (f2 is None) or f1 != f2:
                raise ValueError("line %d: third body on one side only" % no)
            kind = "ELEM"
            eff = {}
            if t1 is not None:
                kind = "THREEBODY"
            if f1 is not None:
                kind = "LINDEMANN"
                if f1.upper() != "M":
                    if f1 not in nameset:
                        raise ValueError("line %d: unknown collider %s" % (no, f1))
                    eff = {n: (1.0 if n == f1 else 0.0) for n in names}
            cur = Reaction(reac, prod, A, b, E * efac, kind, op != "=>", eff)
            reactions.append(cur)
            continue
        if cur is None:
            raise ValueError("line %d: auxiliary data before the first reaction" % no)
        for m in re.finditer(r"([A-Za-z][A-Za-z0-9_()*,\-]*)\s*(?:/([^/]*)/)?", text):
            key, val = m.group(1), m.group(2)
            ku = key.upper()
            if ku in ("DUPLICATE", "DUP"):
                continue
            if ku in _UNSUPPORTED:
                raise ValueError("line %d: %s is not supported" % (no, ku))
            if val is None:
                raise ValueError("line %d: unexpected %r" % (no, key))
            nums = [float(v.replace("D", "E")) for v in val.split()]
            if ku == "LOW":
                if cur.kind not in ("LINDEMANN", "TROE") or len(nums) != 3:
                    raise ValueError("line %d: LOW needs a (+M) reaction and three values" % no)
                cur.low = (nums[0], nums[1], nums[2] * efac)
            elif ku == "TROE":
                if cur.kind not in ("LINDEMANN", "TROE") or len(nums) not in (3, 4):
                    raise ValueError("line %d: TROE needs a (+M) reaction and 3 or 4 values" % no)
                cur.kind = "TROE"
                cur.troe = tuple(nums)
            else:
                if key not in nameset:
                    raise ValueError("line %d: efficiency for unknown species %s" % (no, key))
                if cur.kind == "ELEM":
                    raise ValueError("line %d: efficiencies on a reaction without +M" % no)
                if len(nums) != 1:
                    raise ValueError("line %d: efficiency needs one value" % no)
                cur.eff[key] = nums[0]
    for r in reactions:
        if r.kind in ("LINDEMANN", "TROE") and r.low is None:
            raise ValueError("falloff reaction without LOW")
    return Mechanism(elements, species, reactions)


def _nasa_record(s: Species) -> str:
    comp = list(s.comp.items())
    if len(comp) > 4:
        raise ValueError("species %s has more than four elements" % s.name)
    cf = "".join("%-2s%3d" % (e.upper(), c) for e, c in comp).ljust(20)
    l1 = "%-18s%6s%s%s%10.3f%10.3f%8.2f      1" % (s.name, "", cf, "G", s.Tlow, s.Thigh, s.Tmid)
    c = list(s.hi) + list(s.lo)
    fmt = lambda v: "%15.8E" % v
    l2 = "".join(fmt(v) for v in c[0:5]) + "    2"
    l3 = "".join(fmt(v) for v in c[5:10]) + "    3"
    l4 = "".join(fmt(v) for v in c[10:14]) + "                   4"
    return "\n".join((l1, l2, l3, l4))


def write_chemkin(mech: Mechanism) -> str:
    """The mechanism as CHEMKIN-II text with an inline THERMO section (kJ/mol units)."""
    out = ["ELEMENTS", " ".join(e.upper() for e in mech.elements), "END", "SPECIES"]
    out += [" ".join(s.name for s in mech.species[i:i + 8]) for i in range(0, mech.K, 8)]
    out += ["END", "THERMO ALL", "   200.000  1000.000  6000.000"]
    out += [_nasa_record(s) for s in mech.species]
    out += ["END", "REACTIONS KJOULES/MOLE MOLES"]
    for r in mech.reactions:
        side = lambda lst: " + ".join(("%d %s" % (c, n)) if c != 1 else n for n, c in lst)
        tb = " + M" if r.kind == "THREEBODY" else (" (+M)" if r.kind in ("LINDEMANN", "TROE") else "")
        op = "<=>" if r.reversible else "=>"
        out.append("%s%s %s %s%s   %.17g %.17g %.17g" % (side(r.reac), tb, op, side(r.prod), tb, r.A, r.b, r.E))
        if r.low is not None:
            out.append("   LOW / %.17g %.17g %.17g /" % r.low)
        if r.troe is not None:
            out.append("   TROE / %s /" % " ".join("%.17g" % v for v in r.troe))
        if r.eff:
            out.append("   " + " ".join("%s/%.17g/" % (n, a) for n, a in r.eff.items()))
    out.append("END")
    return "\n".join(out) + "\n"


def main(argv=None) -> int:
    """python -m paper_2508_16105_gb300.chemkin MECH [THERMO]: print the RDEMECH 1 text."""
    import sys
    args = sys.argv[1:] if argv is None else argv
    if not 1 <= len(args) <= 2:
        sys.stderr.write("usage: python -m paper_2508_16105_gb300.chemkin MECH [THERMO]\n")
        return 2
    with open(args[0]) as f:
        mech_text = f.read()
    thermo_text = None
    if len(args) == 2:
        with open(args[1]) as f:
            thermo_text = f.read()
    sys.stdout.write(read_chemkin(mech_text, thermo_text).to_text())
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
