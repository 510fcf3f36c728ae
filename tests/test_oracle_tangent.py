"""Pins for the oracle's exact tangent of the frozen-step map (complex step).

- First-order isomerisation A -> B at fixed T: the tangent of Y_A(dt) with
  respect to ln A, E, Y_A0 and T0 equals the derivative of Y_A0 exp(-k dt),
  k = A T^b exp(-E/(R_u T)), to the integration tolerance.
- On the 9-species mechanism the tangent agrees with central finite
  differences of the real frozen-step replay (norm-wise, within the FD error).
- It is linear in the direction.
"""
import numpy as np

import oracle
from paper_2508_16105_gb300 import synth

RU = 8.31446261815324


def test_first_order_closed_form():
    A, b, E, T, p = 2.0e6, 0.5, 50.0, 1500.0, 2.0e5
    mech = synth.isomer_mechanism(A=A, b=b, E=E)
    o = oracle.Oracle(mech.to_text())
    k = A * T ** b * np.exp(-E * 1e3 / (RU * T))
    dt = 1.3 / k
    y0 = np.array([0.6, 0.1, 0.3, T])
    rc, y1, steps = oracle.record(o, p, y0, dt, oracle.default_opts(rtol=1e-11, atol=1e-16))
    assert rc == 0 and len(steps) > 10
    YA = 0.6 * np.exp(-k * dt)
    _, d = oracle.tangent(o, p, y0, steps, dlnA=[1.0])
    assert abs(d[0] - (-k * dt * YA)) < 1e-8 * abs(k * dt * YA)
    assert abs(d[1] + d[0]) < 1e-14          # mass conserved
    _, d = oracle.tangent(o, p, y0, steps, dE=[1.0])
    assert abs(d[0] - (k * dt * YA / (RU * T))) < 1e-8 * abs(k * dt * YA / (RU * T))
    _, d = oracle.tangent(o, p, y0, steps, dy0=[1.0, 0, 0, 0])
    assert abs(d[0] - np.exp(-k * dt)) < 1e-9
    _, d = oracle.tangent(o, p, y0, steps, dy0=[0, 0, 0, 1.0])
    dkdT = k * (b / T + E * 1e3 / (RU * T * T))
    assert abs(d[0] - (-YA * dt * dkdT)) < 1e-8 * abs(YA * dt * dkdT)
    assert abs(d[3] - 1.0) < 1e-14           # isothermal: T0 carries through


def _fd(o, p, y0, steps, dy0, dlnA, dE, h):
    _, yp = oracle.replay(o, p, y0 + h * dy0, steps, dlnA=h * dlnA, dE=h * dE)
    _, ym = oracle.replay(o, p, y0 - h * dy0, steps, dlnA=-h * dlnA, dE=-h * dE)
    return (yp - ym) / (2 * h)


def test_against_finite_differences(h2mech, h2oracle):
    o = h2oracle
    cells = synth.uniform_cells(h2mech, 3, seed=1001)
    for i in range(cells.n):
        y0 = np.append(cells.Y[:, i], cells.T[i])
        p = cells.p[i]
        rc, _, steps = oracle.record(o, p, y0, 1e-8)
        assert rc == 0
        for trial in range(3):
            u = synth.uniform(40 + i, "dir%d" % trial, 10 + 42) - 0.5
            dy0 = u[:10] * np.append(np.full(9, 1e-3), 10.0)
            dlnA = u[10:31] * 0.1
            dE = u[31:52] * 100.0
            _, t = oracle.tangent(o, p, y0, steps, dy0=dy0, dlnA=dlnA, dE=dE)
            fd = _fd(o, p, y0, steps, dy0, dlnA, dE, 1e-4)
            scale = np.abs(t) + np.array([1e-12] * 9 + [1e-6])
            assert (np.abs(t - fd) / (np.abs(t).max(keepdims=True) + scale)).max() < 1e-6


def test_linear_in_direction(h2mech, h2oracle):
    o = h2oracle
    cells = synth.uniform_cells(h2mech, 1, seed=1001)
    y0 = np.append(cells.Y[:, 0], cells.T[0])
    rc, _, steps = oracle.record(o, cells.p[0], y0, 1e-8)
    a = synth.uniform(7, "a", 10) - 0.5
    b = synth.uniform(7, "b", 21) - 0.5
    _, ta = oracle.tangent(o, cells.p[0], y0, steps, dy0=a)
    _, tb = oracle.tangent(o, cells.p[0], y0, steps, dlnA=b)
    _, tab = oracle.tangent(o, cells.p[0], y0, steps, dy0=2 * a, dlnA=-3 * b)
    assert np.abs(tab - (2 * ta - 3 * tb)).max() <= 1e-12 * np.abs(tab).max()
