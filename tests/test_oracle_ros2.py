"""Pins for the second method, ROS2 (2 stages, order 2, embedded order 1, L-stable).

The oracle stores it in the transformed form; converted back to the classical
parameters of Hairer & Wanner (Solving ODEs II, Section IV.7), the order
conditions of their Table 7.1 must hold through order 2 for the main method and
order 1 for the embedded one (which must differ at order 2, else its estimate
vanishes), the method must be L-stable and A-stable, and the fixed-step global
error on a problem with a closed-form solution must fall with slope 2 (one
local-error estimate with slope 2 per halving of h, i.e. order 1 + 1).
"""
import numpy as np
import pytest

import oracle
from paper_2508_16105_gb300 import synth

RU = 8.31446261815324
ROS2 = oracle.METHOD_ROS2


def classical():
    s, g, a, c, m, e, qhat = oracle.tableau_method(ROS2)
    Ginv = np.diag(np.full(s, 1.0 / g)) - np.tril(c, -1)
    G = np.linalg.inv(Ginv)
    alpha = np.tril(a, -1) @ G
    return s, g, alpha, G, m @ G, (m - e) @ G, qhat


def test_shape_and_gamma():
    s, g, alpha, G, b, bhat, qhat = classical()
    assert s == 2 and qhat == 1
    assert np.allclose(np.diag(G), g) and abs(g - (1 - 1 / np.sqrt(2))) < 1e-16


def test_order_conditions():
    s, g, alpha, G, b, bhat, qhat = classical()
    beta_i = np.tril(alpha + G, -1).sum(1)
    assert abs(b.sum() - 1) < 1e-15 and abs(b @ beta_i - (0.5 - g)) < 1e-15     # order 2
    assert abs(bhat.sum() - 1) < 1e-15                                            # embedded order 1
    assert abs(bhat @ beta_i - (0.5 - g)) > 1e-2                                  # ... and not 2
    a_i = alpha.sum(1)
    assert abs(b @ a_i ** 2 - 1 / 3) > 1e-3                                       # not order 3


def stability(z, b, alpha, G):
    return 1.0 + z * b @ np.linalg.solve(np.eye(len(b)) - z * (alpha + G), np.ones(len(b)))


def test_L_and_A_stable():
    s, g, alpha, G, b, bhat, qhat = classical()
    assert abs(1.0 - b @ np.linalg.solve(alpha + G, np.ones(s))) < 1e-14          # R(inf) = 0
    for y in np.concatenate([np.logspace(-3, 5, 60), -np.logspace(-3, 5, 60)]):
        assert abs(stability(1j * y, b, alpha, G)) <= 1.0 + 1e-12
    for z in (1e-2, -1e-2, 2e-2j):
        assert abs(stability(z, b, alpha, G) - np.exp(z)) < 5 * abs(z) ** 3         # order 2


def test_fixed_step_order2_on_dimerisation():
    """2A -> B at fixed T: 1/Y - ln Y = 1/Y0 - ln Y0 + kappa t (closed form of the oracle's model)."""
    A, T, p = 3.0e9, 900.0, 2.0e5
    mech = synth.dimer_mechanism(A=A, b=0.0, E=0.0)
    o = oracle.Oracle(mech.to_text())
    kappa = 4 * A * 1e-6 * p / (RU * T)
    t_end = 2.0 / kappa

    def exact(y0, t):
        from scipy.optimize import brentq
        c = 1 / y0 - np.log(y0) + kappa * t
        return brentq(lambda y: 1 / y - np.log(y) - c, 1e-12, 1.0)

    errs, ests = [], []
    for n in (20, 40, 80, 160):
        h = t_end / n
        y = np.array([0.9, 0.1, T])
        for i in range(n):
            rc, y, e = o.fixed_step(p, y, h, method=ROS2)
            assert rc == 0
            if i == 0:
                ests.append(abs(e[0]))
        errs.append(abs(y[0] - exact(0.9, t_end)))
    slopes = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert (slopes > 1.8).all() and (slopes < 2.3).all(), slopes
    est_slopes = np.log2(np.array(ests[:-1]) / np.array(ests[1:]))
    assert (est_slopes > 1.8).all(), est_slopes


def test_adaptive_ros2_conserves_and_agrees(h2mech, h2oracle):
    """Adaptive ROS2 at rtol 1e-6 on the H2 mechanism: mass conserved, and within a few
    rtol of RODAS3 at rtol 1e-10 (both integrate the same ODE)."""
    cells = synth.uniform_cells(h2mech, 8, seed=1001)
    T2, Y2, st2, na2, nr2, _ = h2oracle.advance(cells.p, cells.T, cells.Y, 1e-8,
                                               oracle.default_opts(rtol=1e-6, atol=1e-10, method=ROS2))
    T3, Y3, st3, na3, nr3, _ = h2oracle.advance(cells.p, cells.T, cells.Y, 1e-8,
                                               oracle.default_opts(rtol=1e-10, atol=1e-14))
    assert (st2 == 0).all() and (st3 == 0).all()
    assert np.abs(Y2.sum(0) - cells.Y.sum(0)).max() < 1e-12
    assert np.abs(T2 / T3 - 1).max() < 2e-5, np.abs(T2 / T3 - 1).max()
    assert na2.sum() > na3.sum() / 10          # a low-order method takes real steps


def test_adaptive_ros2_vs_radau(h2mech, h2oracle):
    """Adaptive ROS2 at rtol 1e-8 against scipy's Radau IIA at rtol 1e-12 on the same
    right-hand side: an integrator that shares nothing with the oracle's Rosenbrock code
    bounds its global error (the bounds of the RODAS3 pin)."""
    from scipy.integrate import solve_ivp
    cells = synth.uniform_cells(h2mech, 3, seed=1001)
    T, Y, st, na, nr, _ = h2oracle.advance(cells.p, cells.T, cells.Y, 1e-8,
                                           oracle.default_opts(rtol=1e-8, method=ROS2))
    assert (st == 0).all()
    for i in range(cells.n):
        p = cells.p[i]
        y0 = np.append(cells.Y[:, i], cells.T[i])
        sol = solve_ivp(lambda t, y: h2oracle.rhs(p, y), (0, 1e-8), y0, method="Radau",
                        rtol=1e-12, atol=1e-18, jac=lambda t, y: h2oracle.jac(p, y)[1])
        ref = sol.y[:, -1]
        assert abs(T[i] - ref[-1]) / ref[-1] < 1e-7
        assert np.abs(Y[:, i] - ref[:-1]).max() < 2e-10
