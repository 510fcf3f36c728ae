"""Invariants of the constant-pressure reactor, checked on the oracle.

Element-balanced reactions conserve mass and elements: sum_k Y_k = 1 and
sum_k E_ek Y_k / W_k are constant along the exact solution and, because every
Rosenbrock increment is a combination of f and of solves with a Jacobian whose
columns keep those sums, along the numerical one to rounding.  The energy
equation of an adiabatic constant-pressure reactor conserves the mixture's
specific enthalpy sum_k Y_k H_k(T) / W_k to the integration tolerance.
"""
import numpy as np

from paper_2508_16105_gb300 import synth

RU = 8.31446261815324


def nasa_h(coeffs, T):
    a = coeffs
    return RU * T * (a[0] + a[1] * T / 2 + a[2] * T ** 2 / 3 + a[3] * T ** 3 / 4 + a[4] * T ** 4 / 5 + a[5] / T)


def test_invariants_h2_mechanism(h2mech, h2oracle):
    cells = synth.uniform_cells(h2mech, 24, seed=1001)
    T, Y, st, na, nr, _ = h2oracle.advance(cells.p, cells.T, cells.Y, 1e-8, threads=4)
    assert (st == 0).all()
    assert np.abs(Y.sum(0) - 1.0).max() < 1e-12
    W = h2mech.W_array() / 1000.0
    comp = np.array([[s.comp.get(e, 0) for e in h2mech.elements] for s in h2mech.species], float)
    el0 = comp.T @ (cells.Y / W[:, None])
    el1 = comp.T @ (Y / W[:, None])
    assert (np.abs(el1 - el0) / np.abs(el0).max(0)).max() < 1e-12
    # specific enthalpy (J/kg); coefficients identical in both ranges for this mechanism
    for i in range(cells.n):
        h0 = sum(cells.Y[k, i] * nasa_h(s.lo, cells.T[i]) / W[k] for k, s in enumerate(h2mech.species))
        h1 = sum(Y[k, i] * nasa_h(s.lo, T[i]) / W[k] for k, s in enumerate(h2mech.species))
        cp_scale = 2000.0 * T[i]   # J/kg: a typical |c_p T|
        assert abs(h1 - h0) / cp_scale < 1e-7
    # the temperature actually moves: the invariant is not trivially satisfied
    assert np.abs(T - cells.T).max() > 1.0


def test_sum_of_rhs_is_zero(h2mech, h2oracle):
    cells = synth.uniform_cells(h2mech, 16, seed=7)
    for i in range(cells.n):
        y = np.append(cells.Y[:, i], cells.T[i])
        f = h2oracle.rhs(cells.p[i], y)
        scale = np.abs(f[:-1]).max()
        assert abs(f[:-1].sum()) <= 1e-13 * scale
