"""Pins for the Troe falloff blending (Gilbert, Luther & Troe 1983, in the form
of the CHEMKIN theory manual): log10 F = log10 Fcent / (1 + X^2) with
X = (log10 Pr + c) / (n - 0.14 (log10 Pr + c)), c = -0.4 - 0.67 log10 Fcent,
n = 0.75 - 1.27 log10 Fcent.

Structural special values checked through the oracle's k_f:
  - Fcent = 1 (a = 0, T*** -> inf) reduces Troe to Lindemann;
  - at log10 Pr = -c, X = 0 and F = Fcent exactly;
  - at log10 Pr + c = n/(1+d) or -n/(1-d), X^2 = 1 and log10 F = log10 Fcent / 2.
"""
import numpy as np
import pytest

import oracle
from paper_2508_16105_gb300 import synth

RU = 8.31446261815324


def kf_of(mech, T, p):
    o = oracle.Oracle(mech.to_text())
    y = np.array([0.6, 0.1, 0.3, T])
    kf, kr, q = o.rates(p, y)
    return kf[0]


def arrh(A, b, E, T):
    return A * T ** b * np.exp(-E * 1e3 / (RU * T))


def fcent(a, T3, T1, T2, T):
    v = (1 - a) * np.exp(-T / T3) + a * np.exp(-T / T1)
    return v + (np.exp(-T2 / T) if T2 is not None else 0.0)


def test_troe_unit_fcent_is_lindemann():
    T, p = 1300.0, 5.0e4
    kinf_p, k0_p = (3.0e5, 0.2, 30.0), (4.0e12, -0.5, 10.0)
    lind = synth.isomer_mechanism(kind="LINDEMANN", A=kinf_p[0], b=kinf_p[1], E=kinf_p[2], low=k0_p)
    troe = synth.isomer_mechanism(kind="TROE", A=kinf_p[0], b=kinf_p[1], E=kinf_p[2], low=k0_p,
                                  troe=(0.0, 1e300, 1.0))
    assert abs(kf_of(troe, T, p) / kf_of(lind, T, p) - 1) < 1e-14


def _pr_target(u_offset, a, T3, T1, T2, T):
    Fc = fcent(a, T3, T1, T2, T)
    Lc = np.log10(Fc)
    c = -0.4 - 0.67 * Lc
    return 10.0 ** (-c + u_offset), Fc


@pytest.mark.parametrize("T2", [None, 4000.0])
@pytest.mark.parametrize("which", ["center", "upper_half", "lower_half"])
def test_troe_special_points(which, T2):
    T, p = 1000.0, 1.0e5
    a, T3, T1 = 0.6, 150.0, 2500.0
    Fc = fcent(a, T3, T1, T2, T)
    Lc = np.log10(Fc)
    n, d = 0.75 - 1.27 * Lc, 0.14
    u = {"center": 0.0, "upper_half": n / (1 + d), "lower_half": -n / (1 - d)}[which]
    Pr, _ = _pr_target(u, a, T3, T1, T2, T)
    # choose A0 so that k0 [M] / kinf = Pr exactly at this state
    kinf_p = (3.0e5, 0.0, 0.0)
    M = p / (RU * T)
    A0_si = Pr * kinf_p[0] / M
    troe = (a, T3, T1) if T2 is None else (a, T3, T1, T2)
    mech = synth.isomer_mechanism(kind="TROE", A=kinf_p[0], b=0.0, E=0.0, low=(A0_si * 1e6, 0.0, 0.0), troe=troe)
    F_expected = Fc if which == "center" else 10.0 ** (Lc / 2)
    k_expected = kinf_p[0] * Pr / (1 + Pr) * F_expected
    assert abs(kf_of(mech, T, p) / k_expected - 1) < 1e-12
