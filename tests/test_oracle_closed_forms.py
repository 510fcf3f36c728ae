"""Closed-form pins for the oracle's kinetics and integrator.

Each mechanism here reduces the constant-pressure reactor to an ODE with a known
solution: isomerisation A -> B (first order, exp(-k t)); the reversible case
with K_c = 1 (relaxation to the mean at rate 2k); a third-body reaction whose
[M] = p/(R_u T) with unit efficiencies; Lindemann falloff k = k_inf Pr/(1+Pr);
and dimerisation 2A -> B, whose constant-pressure solution satisfies
1/Y - ln Y = 1/Y0 - ln Y0 + 4 k p/(R_u T) t.  Rate constants are
k = A T^b exp(-E/(R_u T)) with A converted from mol-cm-s to SI by 1e-6 per
order above one.
"""
import numpy as np
import pytest

import oracle
from paper_2508_16105_gb300 import synth

RU = 8.31446261815324
TIGHT = oracle.default_opts(rtol=1e-11, atol=1e-16)


def arrh(A, b, E_kJ, T):
    return A * T ** b * np.exp(-E_kJ * 1e3 / (RU * T))


def run(mech, p, T, Y, dt, opts=TIGHT):
    o = oracle.Oracle(mech.to_text())
    Tn, Yn, st, na, nr, _ = o.advance(np.array([p]), np.array([T]), np.array(Y, float).reshape(-1, 1), dt, opts)
    assert st[0] == 0
    return Tn[0], Yn[:, 0]


@pytest.mark.parametrize("b,E", [(0.0, 0.0), (0.5, 50.0), (-0.7, 120.0)])
def test_irreversible_first_order(b, E):
    T, p = 1500.0, 2.0e5
    A = 2.0e6 if E < 100 else 2.0e9
    mech = synth.isomer_mechanism(A=A, b=b, E=E)
    k = arrh(A, b, E, T)
    dt = 1.5 / k
    Y0 = [0.6, 0.1, 0.3]
    Tn, Y = run(mech, p, T, Y0, dt)
    assert abs(Y[0] - 0.6 * np.exp(-k * dt)) < 1e-10 * 0.6
    assert abs(Y[1] - (0.7 - 0.6 * np.exp(-k * dt))) < 1e-10
    assert abs(Y[2] - 0.3) < 1e-15
    assert abs(Tn - T) < 1e-9


def test_reversible_equal_thermo():
    T, p = 1200.0, 1.0e5
    A, b, E = 5.0e5, 0.3, 10.0
    mech = synth.isomer_mechanism(reversible=True, A=A, b=b, E=E)
    k = arrh(A, b, E, T)
    for kt in (0.2, 1.0, 4.0):
        Tn, Y = run(mech, p, T, [0.7, 0.0, 0.3], kt / k)
        mean = 0.35
        assert abs(Y[0] - (mean + (0.7 - mean) * np.exp(-2 * kt))) < 1e-10
        assert abs(Y[0] + Y[1] - 0.7) < 1e-14


@pytest.mark.parametrize("eff", [None, {"X2": 2.5}])
def test_three_body_concentration(eff):
    T, p = 1500.0, 3.0e5
    A, b, E = 2.0e10, 0.0, 20.0
    mech = synth.isomer_mechanism(kind="THREEBODY", A=A, b=b, E=E)
    if eff:
        mech.reactions[0].eff = dict(eff)
    Y0 = np.array([0.6, 0.1, 0.3])
    # all species have W = 20 g/mol: rho = p W / (R T); c_k = rho Y_k / W
    rho = p * 0.020 / (RU * T)
    c = rho * Y0 / 0.020
    M = c.sum() if not eff else c[0] + c[1] + 2.5 * c[2]
    if not eff:
        assert abs(M - p / (RU * T)) < 1e-12 * M
    k = arrh(A, b, E, T) * 1e-6 * M
    dt = 2.0 / k
    Tn, Y = run(mech, p, T, Y0, dt)
    assert abs(Y[0] - 0.6 * np.exp(-k * dt)) < 1e-10 * 0.6


def test_lindemann_falloff():
    T, p = 1300.0, 5.0e4
    kinf_p = (3.0e5, 0.2, 30.0)
    k0_p = (4.0e12, -0.5, 10.0)
    mech = synth.isomer_mechanism(kind="LINDEMANN", A=kinf_p[0], b=kinf_p[1], E=kinf_p[2], low=k0_p)
    M = p / (RU * T)
    kinf = arrh(*kinf_p, T)
    k0 = arrh(*k0_p, T) * 1e-6
    Pr = k0 * M / kinf
    k = kinf * Pr / (1 + Pr)
    assert 0.05 < Pr < 20  # genuinely in the falloff region
    dt = 1.0 / k
    Tn, Y = run(mech, p, T, [0.6, 0.1, 0.3], dt)
    assert abs(Y[0] - 0.6 * np.exp(-k * dt)) < 1e-10 * 0.6


def test_dimerisation_second_order():
    T, p = 900.0, 2.0e5
    A, b, E = 3.0e9, 0.4, 15.0
    mech = synth.dimer_mechanism(A=A, b=b, E=E)
    k = arrh(A, b, E, T) * 1e-6           # second order: cm^3 -> m^3
    kappa = 4.0 * k * p / (RU * T)
    Y0 = 0.9
    for kt in (0.3, 2.0):
        t = kt / kappa
        Tn, Y = run(mech, p, T, [Y0, 1 - Y0], t)
        rhs = 1 / Y0 - np.log(Y0) + kappa * t
        y = Y0
        for _ in range(60):               # Newton on g(y) = 1/y - ln y - rhs
            g = 1 / y - np.log(y) - rhs
            y -= g / (-1 / y ** 2 - 1 / y)
        assert abs(Y[0] - y) < 1e-10
        assert abs(Tn - T) < 1e-9
