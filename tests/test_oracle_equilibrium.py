"""HP-equilibrium pin for the oracle's equilibrium constants and energy equation.

Mechanism: H2 + M <=> 2 H + M with inert N2.  Integrated to t = 1 s at constant
p, the reactor must reach the constant-(H, p) equilibrium.  That state is found
here without kinetics or K_c: for each T the extent of dissociation minimising
G/(R_u T) = sum_k n_k (g_k(T) + ln(x_k p / P_std)) is located by a fine scan and
golden-section search, and T is found by bisection on the mixture enthalpy.
"""
import numpy as np

import oracle
from paper_2508_16105_gb300 import synth

RU = 8.31446261815324
PSTD = 101325.0


def g_RT(a, T):
    h = a[0] + a[1] * T / 2 + a[2] * T ** 2 / 3 + a[3] * T ** 3 / 4 + a[4] * T ** 4 / 5 + a[5] / T
    s = a[0] * np.log(T) + a[1] * T + a[2] * T ** 2 / 2 + a[3] * T ** 3 / 3 + a[4] * T ** 4 / 4 + a[6]
    return h - s, h


def moles(n0, xi):
    return np.array([n0[0] - xi, n0[1] + 2 * xi, n0[2]])


def gibbs(mech, n0, T, p, xi):
    n = moles(n0, xi)
    g = np.array([g_RT(s.lo, T)[0] for s in mech.species])
    x = n / n.sum()
    with np.errstate(divide="ignore", invalid="ignore"):
        terms = np.where(n > 0, n * (g + np.log(x * p / PSTD)), 0.0)
    return terms.sum()


def xi_star(mech, n0, T, p):
    lo, hi = -n0[1] / 2 + 1e-300, n0[0]
    grid = np.linspace(lo, hi, 2001)[1:-1]
    vals = [gibbs(mech, n0, T, p, x) for x in grid]
    i = int(np.argmin(vals))
    a, b = grid[max(i - 1, 0)], grid[min(i + 1, len(grid) - 1)]
    phi = (np.sqrt(5) - 1) / 2
    for _ in range(200):
        c, d = b - phi * (b - a), a + phi * (b - a)
        if gibbs(mech, n0, T, p, c) < gibbs(mech, n0, T, p, d):
            b = d
        else:
            a = c
    return 0.5 * (a + b)


def enthalpy(mech, n, T):
    return sum(n[k] * RU * T * g_RT(s.lo, T)[1] for k, s in enumerate(mech.species))


def test_hp_equilibrium():
    mech = synth.dissociation_mechanism()
    W = mech.W_array() / 1000.0
    p, T0 = 101325.0, 4200.0
    Y0 = np.array([0.25, 0.0, 0.75])
    n0 = Y0 / W                   # moles per kg of mixture
    H0 = enthalpy(mech, n0, T0)
    lo, hi = 1500.0, T0
    for _ in range(80):
        T = 0.5 * (lo + hi)
        n = moles(n0, xi_star(mech, n0, T, p))
        if enthalpy(mech, n, T) > H0:
            hi = T
        else:
            lo = T
    Teq = 0.5 * (lo + hi)
    neq = moles(n0, xi_star(mech, n0, Teq, p))
    Yeq = neq * W

    o = oracle.Oracle(mech.to_text())
    T1, Y1, st, na, nr, _ = o.advance(np.array([p]), np.array([T0]), Y0.reshape(-1, 1), 1.0,
                                      oracle.default_opts(rtol=1e-10, atol=1e-14))
    assert st[0] == 0
    assert Yeq[1] > 1e-3                         # substantial dissociation: a real test
    assert abs(T1[0] - Teq) / Teq < 1e-6
    assert np.abs(Y1[:, 0] - Yeq).max() < 1e-8
