"""Seeded input generators: determinism, element balance, compositions."""
import numpy as np

from paper_2508_16105_gb300 import synth


def test_uniform_reproducible_and_offset():
    a = synth.uniform(3, "x", 100)
    b = synth.uniform(3, "x", 40, offset=60)
    assert np.array_equal(a[60:], b)
    assert not np.array_equal(a, synth.uniform(4, "x", 100))
    assert 0.0 <= a.min() and a.max() < 1.0
    assert abs(synth.uniform(1, "big", 200000).mean() - 0.5) < 5e-3


def test_mechanisms_element_balanced():
    for mech in (synth.h2_air_mechanism(), synth.robertson_mechanism(), synth.dissociation_mechanism(),
                 synth.dimer_mechanism(), synth.isomer_mechanism()):
        for r in mech.reactions:
            bal = {}
            for n, c in r.reac:
                for e, v in mech.species[mech.index(n)].comp.items():
                    bal[e] = bal.get(e, 0) - c * v
            for n, c in r.prod:
                for e, v in mech.species[mech.index(n)].comp.items():
                    bal[e] = bal.get(e, 0) + c * v
            assert all(v == 0 for v in bal.values()), r


def test_h2_mechanism_shape():
    m = synth.h2_air_mechanism()
    assert (m.K, m.R) == (9, 21)
    assert sum(r.kind == "THREEBODY" for r in m.reactions) == 3
    assert all(r.reversible for r in m.reactions)
    for r in m.reactions:
        assert 1e9 <= r.A <= 1e17 and -1 <= r.b <= 1 and 0 <= r.E <= 200
    assert m.to_text() == synth.h2_air_mechanism().to_text()


def test_cell_states():
    m = synth.h2_air_mechanism()
    c = synth.uniform_cells(m, 1000, seed=1001)
    assert np.abs(c.Y.sum(0) - 1).max() < 1e-14
    assert c.T.min() >= 800 and c.T.max() <= 3000
    f = synth.field_cells(m, 10000, seed=1002)
    assert np.bincount(f.cls).tolist() == [9000, 500, 500]
    assert np.abs(f.Y.sum(0) - 1).max() < 1e-14
    fresh = f.T[f.cls == 0]
    assert fresh.min() >= 300 and fresh.max() <= 600
    assert (f.Y >= 0).all()
