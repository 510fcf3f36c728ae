"""NASA-7 thermodynamics of the oracle.

Pins: dH/dT = Cp and dS/dT = Cp/T (finite differences) catch a wrong power or
divisor in any of the three polynomials; flat fits (a2..a5 = 0) have the closed
forms Cp/R = a1, H/RT = a1 + a6/T, S/R = a1 ln T + a7; the low range applies
below Tmid and the high range at and above it.
"""
import numpy as np

import oracle
from paper_2508_16105_gb300 import synth


def test_derivative_relations(h2mech, h2oracle):
    for k in range(h2mech.K):
        for T in (300.0, 800.0, 1500.0, 2500.0, 3500.0):
            d = 1e-5 * T
            cp, h, s = h2oracle.thermo(k, T)
            _, hp, sp = h2oracle.thermo(k, T + d)
            _, hm, sm = h2oracle.thermo(k, T - d)
            dH = ((T + d) * hp - (T - d) * hm) / (2 * d)     # d(H/R)/dT
            dS = (sp - sm) / (2 * d)
            assert abs(dH - cp) < 1e-8 * cp
            assert abs(dS - cp / T) < 1e-8 * cp / T


def test_flat_fits():
    mech = synth.isomer_mechanism()
    o = oracle.Oracle(mech.to_text())
    a1, a6, a7 = 3.5, -1000.0, 5.0
    for T in (250.0, 1000.0, 4000.0):
        cp, h, s = o.thermo(0, T)
        assert cp == a1
        assert abs(h - (a1 + a6 / T)) < 1e-15 * abs(h)
        assert abs(s - (a1 * np.log(T) + a7)) < 1e-14 * abs(s)


def test_range_selection_and_continuity():
    mech = synth.two_range_mechanism()
    o = oracle.Oracle(mech.to_text())
    lo, hi = mech.species[0].lo, mech.species[0].hi
    cp_lo = lambda T: lo[0] + lo[1] * T
    cp_hi = lambda T: hi[0] + hi[1] * T
    assert abs(o.thermo(0, 500.0)[0] - cp_lo(500.0)) < 1e-13
    assert abs(o.thermo(0, 1500.0)[0] - cp_hi(1500.0)) < 1e-13
    assert abs(o.thermo(0, 1000.0)[0] - cp_hi(1000.0)) < 1e-13   # tie -> high range
    a = o.thermo(0, 1000.0 - 1e-9)
    b = o.thermo(0, 1000.0)
    assert np.allclose(a, b, rtol=1e-10, atol=0)
