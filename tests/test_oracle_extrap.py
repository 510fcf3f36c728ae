"""Pins for the third method: linearly implicit Euler extrapolation of fixed order 3.

A step of size H from y with J = J(y) runs the linearly implicit Euler method
(I/h - J)(y_{i+1} - y_i) = f(y_i) with n = 1, 2, 3 substeps of h = H/n and
extrapolates the three results (Aitken-Neville for an error expansion in powers
of h) to T_33; the error estimate is T_33 - T_32.  Pins:
  - on linear decay y' = -k y (the isomerisation A -> B at fixed T) one step
    multiplies y by the method's stability function R(z), z = -k H, written out
    here from the definition: T_j1 = (1 - z/n_j)^(-n_j), extrapolated.  It
    tends to 0 as z -> -inf (L-stable at infinity), has |R| <= 1 on the negative
    axis (it dips to -0.0135 near z = -7.45), and agrees with exp(z) to order 3;
  - fixed-step global error on the dimerisation closed form falls as H^3, and
    the per-step error estimate as H^3;
  - adaptive runs conserve mass and agree with scipy's Radau IIA at rtol 1e-12
    within the RODAS3 pin's bounds.
"""
import numpy as np

import oracle
from paper_2508_16105_gb300 import synth

RU = 8.31446261815324
EX = oracle.METHOD_EXTRAP


def stability(z):
    n = np.array([1.0, 2.0, 3.0])
    T = np.zeros((3, 3), dtype=complex)
    T[:, 0] = (1.0 - z / n) ** (-n)
    for k in range(1, 3):
        for j in range(k, 3):
            T[j, k] = T[j, k - 1] + (T[j, k - 1] - T[j - 1, k - 1]) / (n[j] / n[j - k] - 1.0)
    return T[2, 2], T[2, 1]


def test_stability_function_one_step():
    T, p = 1500.0, 2.0e5
    A = 2.0e6
    mech = synth.isomer_mechanism(A=A)
    o = oracle.Oracle(mech.to_text())
    k = A                                  # b = 0, E = 0: k = A (1/s)
    for z in (-1e-3, -0.1, -1.0, -7.5, -60.0, -4e3, -1e6):
        H = -z / k
        rc, yn, e = o.fixed_step(p, np.array([0.6, 0.1, 0.3, T]), H, method=EX)
        assert rc == 0
        R, R32 = stability(z)
        assert abs(yn[0] - 0.6 * R.real) <= 1e-13 * 0.6 + 1e-15, (z, yn[0] / 0.6, R)
        assert abs(e[0] - 0.6 * (R - R32).real) <= 1e-12 * 0.6, (z, e[0], R - R32)
        # B gets the increments of solves with I/h - J, whose rounding grows with |z|
        assert abs(yn[1] - (0.7 - 0.6 * R.real)) <= 1e-12 + 1e-15 * abs(z)
    assert abs(stability(-1e12)[0]) < 1e-10                 # R(-inf) = 0
    zs = -np.logspace(-4, 8, 400)
    Rs = np.array([stability(z)[0].real for z in zs])
    assert (np.abs(Rs) <= 1.0).all()                        # A-stable on the negative axis
    assert Rs.min() < 0.0 and Rs.min() > -0.02              # dips to -0.0135 near z = -7.45
    for z in (1e-2, -1e-2, 2e-2j):
        assert abs(stability(z)[0] - np.exp(z)) < 5 * abs(z) ** 4          # order 3


def test_fixed_step_order3_on_dimerisation():
    A, T, p = 3.0e9, 900.0, 2.0e5
    mech = synth.dimer_mechanism(A=A, b=0.0, E=0.0)
    o = oracle.Oracle(mech.to_text())
    kappa = 4 * A * 1e-6 * p / (RU * T)
    t_end = 2.0 / kappa

    def exact(y0, t):
        from scipy.optimize import brentq
        c = 1 / y0 - np.log(y0) + kappa * t
        return brentq(lambda y: 1 / y - np.log(y) - c, 1e-12, 1.0, xtol=1e-15, rtol=1e-15)

    errs, ests = [], []
    for n in (10, 20, 40, 80):
        h = t_end / n
        y = np.array([0.9, 0.1, T])
        for i in range(n):
            rc, y, e = o.fixed_step(p, y, h, method=EX)
            assert rc == 0
            if i == 0:
                ests.append(abs(e[0]))
        errs.append(abs(y[0] - exact(0.9, t_end)))
    slopes = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert (slopes > 2.7).all() and (slopes < 3.4).all(), slopes
    est_slopes = np.log2(np.array(ests[:-1]) / np.array(ests[1:]))
    assert (est_slopes > 2.7).all(), est_slopes


def test_adaptive_extrapolation_vs_radau(h2mech, h2oracle):
    from scipy.integrate import solve_ivp
    cells = synth.uniform_cells(h2mech, 3, seed=1001)
    T, Y, st, na, nr, _ = h2oracle.advance(cells.p, cells.T, cells.Y, 1e-8, oracle.default_opts(rtol=1e-8, method=EX))
    assert (st == 0).all()
    assert np.abs(Y.sum(0) - cells.Y.sum(0)).max() < 1e-12
    for i in range(cells.n):
        p = cells.p[i]
        y0 = np.append(cells.Y[:, i], cells.T[i])
        sol = solve_ivp(lambda t, y: h2oracle.rhs(p, y), (0, 1e-8), y0, method="Radau",
                        rtol=1e-12, atol=1e-18, jac=lambda t, y: h2oracle.jac(p, y)[1])
        ref = sol.y[:, -1]
        assert abs(T[i] - ref[-1]) / ref[-1] < 1e-7
        assert np.abs(Y[:, i] - ref[:-1]).max() < 2e-10
