"""CHEMKIN-II import and export (host side, no GPU).

Round trips of the seeded mechanisms (the 9-species set, the 53-species stress set
with three-body and Troe reactions, and the small test mechanisms) through
write_chemkin / read_chemkin keep every field: exactly, except the NASA-7
coefficients, which the format's 15-character fields carry to 9 significant digits.
The imported mechanism gives the oracle the same source terms.  A hand-written
mechanism exercises the syntax the importer accepts (units, reaction arrows,
coefficients, third bodies, falloff with a named collider, efficiencies, a separate
thermo file), and the unsupported keywords are refused by line.
"""
import numpy as np
import pytest

import oracle
from paper_2508_16105_gb300 import chemkin, synth


def _mechs():
    troe = synth.isomer_mechanism(kind="TROE", reversible=True, A=3e5, b=0.3, E=40.0,
                                  low=(4e12, -0.5, 10.0), troe=(0.4, 300.0, 1800.0, 5000.0))
    troe.reactions[0].eff = {"X2": 2.0, "A": 0.7}
    tb = synth.isomer_mechanism(kind="THREEBODY", reversible=True, A=2e10, b=0.2, E=20.0)
    tb.reactions[0].eff = {"X2": 2.5}
    return {"h2": synth.h2_air_mechanism(16105), "large": synth.large_mechanism(),
            "troe": troe, "threebody": tb, "two_range": synth.two_range_mechanism(),
            "robertson": synth.robertson_mechanism()}


@pytest.mark.parametrize("name", ["h2", "large", "troe", "threebody", "two_range", "robertson"])
def test_round_trip(name):
    m = _mechs()[name]
    back = chemkin.read_chemkin(chemkin.write_chemkin(m))
    assert back.elements == m.elements
    assert [s.name for s in back.species] == [s.name for s in m.species]
    for a, b in zip(m.species, back.species):
        assert a.comp == {e: c for e, c in b.comp.items()}
        assert abs(a.W - b.W) <= 1e-12 * a.W
        assert (a.Tlow, a.Tmid, a.Thigh) == (b.Tlow, b.Tmid, b.Thigh)
        for x, y in zip(list(a.lo) + list(a.hi), list(b.lo) + list(b.hi)):
            assert abs(x - y) <= 6e-9 * abs(x) + 1e-300, (a.name, x, y)
    assert len(back.reactions) == len(m.reactions)
    for r, s in zip(m.reactions, back.reactions):
        assert sorted(r.reac) == sorted(s.reac) and sorted(r.prod) == sorted(s.prod)
        assert (r.A, r.b, r.E, r.kind, r.reversible) == (s.A, s.b, s.E, s.kind, s.reversible)
        assert r.eff == s.eff and r.low == s.low and r.troe == s.troe


@pytest.mark.parametrize("name", ["h2", "large"])
def test_imported_mechanism_gives_the_same_source_terms(name):
    m = _mechs()[name]
    back = chemkin.read_chemkin(chemkin.write_chemkin(m))
    oa, ob = oracle.Oracle(m.to_text()), oracle.Oracle(back.to_text())
    cells = synth.field_cells(m, 16, seed=1013, fractions=(0.25, 0.5, 0.25))
    for i in range(cells.n):
        y = np.append(cells.Y[:, i], cells.T[i])
        fa, fb = oa.rhs(cells.p[i], y), ob.rhs(cells.p[i], y)
        scale = np.abs(fa).max()
        assert np.abs(fa - fb).max() <= 1e-6 * scale, (i, np.abs(fa - fb).max() / scale)


THERMO = """THERMO ALL
   300.000  1000.000  5000.000
AA                      X   2               G   300.000  5000.000             1
 3.50000000E+00 1.00000000E-04 0.00000000E+00 0.00000000E+00 0.00000000E+00    2
-1.00000000E+03 4.00000000E+00 3.40000000E+00 2.00000000E-04 0.00000000E+00    3
 0.00000000E+00 0.00000000E+00-1.05000000E+03 4.10000000E+00                   4
BB                      X   1               G   300.000  5000.000 1200.00     1
 2.50000000E+00 0.00000000E+00 0.00000000E+00 0.00000000E+00 0.00000000E+00    2
 2.00000000E+04 5.00000000E+00 2.50000000E+00 0.00000000E+00 0.00000000E+00    3
 0.00000000E+00 0.00000000E+00 2.00000000E+04 5.00000000E+00                   4
CC                      X   2Y   1          G   300.000  5000.000             1
 4.00000000E+00 0.00000000E+00 0.00000000E+00 0.00000000E+00 0.00000000E+00    2
-5.00000000E+03 3.00000000E+00 4.00000000E+00 0.00000000E+00 0.00000000E+00    3
 0.00000000E+00 0.00000000E+00-5.00000000E+03 3.00000000E+00                   4
DD                      Y   1               G   300.000  5000.000             1
 2.50000000E+00 0.00000000E+00 0.00000000E+00 0.00000000E+00 0.00000000E+00    2
 1.00000000E+04 4.00000000E+00 2.50000000E+00 0.00000000E+00 0.00000000E+00    3
 0.00000000E+00 0.00000000E+00 1.00000000E+04 4.00000000E+00                   4
END
"""

MECH = """! a made-up mechanism over two elements
ELEMENTS
X /10.0/ Y /7.5/
END
SPECIES AA BB CC
DD END
REACTIONS          ! default units: cal/mol
2BB + M = AA + M        1.0E15  -1.0   0.0
   AA/2.5/  CC/0.0/
AA + DD <=> CC          2.0E12   0.5   1000.0   ! comment
DUPLICATE
AA + DD <=> CC          3.0E11   0.0   500.0
DUPLICATE
CC => BB + BB + DD      1.5E13   0.0   2.0E4
AA + DD (+AR) <=> CC (+AR)  1.0E13 0.0 0.0
   LOW / 2.0E18 -1.0 100.0 /
AA (+M) <=> 2 BB (+M)   4.0E14   0.0   5.0E4
   LOW / 1.0E16 0.0 4.0E4 /
   TROE / 0.5 100.0 2000.0 /
END
"""


def test_hand_written_mechanism():
    text = MECH.replace("SPECIES AA BB CC", "SPECIES AA BB CC AR").replace(
        "X /10.0/ Y /7.5/", "X /10.0/ Y /7.5/ AR")
    thermo = THERMO.replace("END\n", """AR                      AR  1               G   300.000  5000.000             1
 2.50000000E+00 0.00000000E+00 0.00000000E+00 0.00000000E+00 0.00000000E+00    2
-7.45000000E+02 4.37000000E+00 2.50000000E+00 0.00000000E+00 0.00000000E+00    3
 0.00000000E+00 0.00000000E+00-7.45000000E+02 4.37000000E+00                   4
END
""")
    m = chemkin.read_chemkin(text, thermo)
    assert m.elements == ["X", "Y", "Ar"]
    assert [s.name for s in m.species] == ["AA", "BB", "CC", "AR", "DD"]     # the SPECIES order
    aa, bb, cc = m.species[0], m.species[1], m.species[2]
    assert aa.comp == {"X": 2} and cc.comp == {"X": 2, "Y": 1}
    assert aa.W == 20.0 and cc.W == 27.5 and m.species[3].W == 39.948
    assert aa.Tmid == 1000.0 and bb.Tmid == 1200.0          # global line, then the record's own
    assert aa.hi[:2] == [3.5, 1e-4] and aa.lo[5:] == [-1050.0, 4.1]
    r = m.reactions
    assert len(r) == 6
    cal = 4.184e-3
    assert r[0].kind == "THREEBODY" and r[0].reac == [("BB", 2)] and r[0].prod == [("AA", 1)]
    assert r[0].eff == {"AA": 2.5, "CC": 0.0} and r[0].reversible
    assert r[1].E == pytest.approx(1000.0 * cal) and r[2].A == 3.0e11     # duplicates kept
    assert not r[3].reversible and r[3].prod == [("BB", 2), ("DD", 1)]
    assert r[4].kind == "LINDEMANN" and r[4].eff == {"AA": 0.0, "BB": 0.0, "CC": 0.0, "DD": 0.0, "AR": 1.0}
    assert r[4].low == (2.0e18, -1.0, pytest.approx(100.0 * cal))
    assert r[5].kind == "TROE" and r[5].troe == (0.5, 100.0, 2000.0) and r[5].prod == [("BB", 2)]
    # every reaction conserves the elements, and the oracle takes the result
    for rx in r:
        for e in m.elements:
            count = lambda side: sum(c * m.species[m.index(n)].comp.get(e, 0) for n, c in side)
            assert count(rx.reac) == count(rx.prod), (rx, e)
    o = oracle.Oracle(m.to_text())
    y = np.array([0.2, 0.2, 0.2, 0.2, 0.2, 1200.0])
    assert np.isfinite(o.rhs(2e5, y)).all()


@pytest.mark.parametrize("units,fac", [("KCAL/MOLE", 4.184), ("JOULES/MOLE", 1e-3), ("KJOULES/MOLE", 1.0),
                                       ("KELVINS", 8.31446261815324e-3)])
def test_energy_units(units, fac):
    text = MECH.replace("REACTIONS          ! default units: cal/mol", "REACTIONS " + units + " MOLES")
    m = chemkin.read_chemkin(text.replace("(+AR)", "(+M)"), THERMO)
    assert m.reactions[3].E == pytest.approx(2.0e4 * fac)


@pytest.mark.parametrize("bad,msg", [
    ("   SRI / 0.5 100.0 2000.0 /", "SRI"),
    ("   REV / 1.0E10 0.0 0.0 /", "REV"),
    ("   PLOG / 1.0 1.0E10 0.0 0.0 /", "PLOG"),
])
def test_unsupported_keywords_are_refused(bad, msg):
    text = MECH.replace("   TROE / 0.5 100.0 2000.0 /", bad).replace("(+AR)", "(+M)")
    with pytest.raises(ValueError, match=msg):
        chemkin.read_chemkin(text, THERMO)


def test_errors():
    with pytest.raises(ValueError, match="unknown species"):
        chemkin.read_chemkin(MECH.replace("CC => BB", "EE => BB").replace("(+AR)", "(+M)"), THERMO)
    with pytest.raises(ValueError, match="no thermo data"):
        chemkin.read_chemkin(MECH.replace("(+AR)", "(+M)"), THERMO.split("DD ")[0] + "END\n")
    with pytest.raises(ValueError, match="MOLECULES"):
        chemkin.read_chemkin(MECH.replace("REACTIONS ", "REACTIONS MOLECULES ").replace("(+AR)", "(+M)"), THERMO)
    with pytest.raises(ValueError, match="non-integer"):
        chemkin.read_chemkin(MECH.replace("2BB + M", "1.5BB + M").replace("(+AR)", "(+M)"), THERMO)


def test_command_line(tmp_path, capsys):
    mech = tmp_path / "mech.inp"
    thermo = tmp_path / "therm.dat"
    mech.write_text(MECH.replace("(+AR)", "(+M)"))
    thermo.write_text(THERMO)
    assert chemkin.main([str(mech), str(thermo)]) == 0
    out = capsys.readouterr().out
    assert out.startswith("RDEMECH 1") and out.rstrip().endswith("END")
    assert chemkin.main([]) == 2
