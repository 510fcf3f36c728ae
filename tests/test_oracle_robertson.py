"""Stiff robustness: Robertson's kinetics written as a mechanism, integrated by
the oracle, against scipy's Radau IIA integrator on the textbook ODE
  y1' = -0.04 y1 + 1e4 y2 y3,  y2' = 0.04 y1 - 1e4 y2 y3 - 3e7 y2^2,  y3' = 3e7 y2^2.
With equal molar masses, identical thermo and p = R_u T the mass fractions equal
the concentrations in mol/m^3 and the temperature stays constant.
"""
import numpy as np
import pytest
from scipy.integrate import solve_ivp

import oracle
from paper_2508_16105_gb300 import synth

RU = 8.31446261815324


def robertson(t, y):
    return [-0.04 * y[0] + 1e4 * y[1] * y[2],
            0.04 * y[0] - 1e4 * y[1] * y[2] - 3e7 * y[1] ** 2,
            3e7 * y[1] ** 2]


def robertson_jac(t, y):
    return [[-0.04, 1e4 * y[2], 1e4 * y[1]],
            [0.04, -1e4 * y[2] - 6e7 * y[1], -1e4 * y[1]],
            [0.0, 6e7 * y[1], 0.0]]


@pytest.mark.parametrize("t_end", [0.4, 40.0, 4.0e3])
def test_robertson(t_end):
    mech = synth.robertson_mechanism()
    o = oracle.Oracle(mech.to_text())
    T = 1000.0
    Y0 = np.array([1.0, 0.0, 0.0])
    T1, Y1, st, na, nr, _ = o.advance(np.array([RU * T]), np.array([T]), Y0.reshape(-1, 1), t_end,
                                      oracle.default_opts(rtol=1e-10, atol=1e-16))
    assert st[0] == 0
    ref = solve_ivp(robertson, (0, t_end), Y0, method="Radau", rtol=1e-13, atol=1e-20,
                    jac=robertson_jac).y[:, -1]
    y = Y1[:, 0]
    assert abs(y.sum() - 1.0) < 1e-12
    assert abs(y[0] - ref[0]) < 1e-8 * ref[0]
    assert abs(y[2] - ref[2]) < 1e-8 * max(ref[2], 1e-6)
    assert abs(y[1] - ref[1]) < 1e-7 * ref[1]
    assert abs(T1[0] - T) < 1e-9
