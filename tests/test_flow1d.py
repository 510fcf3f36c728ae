"""The toy 1D flow that hosts the chemistry step in an operator split (no GPU).

Pins of the transport (the chemistry operator is tested on its own elsewhere):
  - a closed tube conserves the mass of every species and the total energy to
    rounding over 200 steps (reflecting walls pass no mass or energy flux);
  - a shock-tube problem (the same cold mixture at 10:1 pressure) sends its shock
    at the speed of the exact Riemann solution for a perfect gas with the
    mixture's gamma (Toro's pressure function solved by Newton's method): the
    numerical shock (where p crosses the mean of p* and p_R) lies within 3 cells
    and 1 % of the exact position.
"""
import numpy as np

from paper_2508_16105_gb300 import flow1d, synth


def _air(mech, n):
    names = [s.name for s in mech.species]
    Y = np.zeros((len(names), n))
    Y[names.index("O2")] = 0.233
    Y[names.index("N2")] = 0.767
    return Y


def _riemann_tube(n):
    mech = synth.h2_air_mechanism(16105)
    x = (np.arange(n) + 0.5) / n
    p = np.where(x < 0.5, 1.0e6, 1.0e5)
    T = np.full(n, 300.0)
    return mech, flow1d.Tube(mech, p, T, _air(mech, n), length=1.0)


def test_closed_tube_conserves_mass_and_energy():
    mech, tube = _riemann_tube(200)
    m0, e0, y0 = tube.rho.sum(), tube.E.sum(), tube.rhoY.sum(axis=1)
    dt = 0.4 * tube.dx / tube.max_wave_speed()
    for _ in range(200):
        tube.step(dt)
    assert abs(tube.rho.sum() - m0) <= 1e-12 * m0
    assert abs(tube.E.sum() - e0) <= 1e-12 * abs(e0)   # E includes formation enthalpies: may be negative
    assert np.abs(tube.rhoY.sum(axis=1) - y0).max() <= 1e-12 * m0


def _exact_shock_speed(gamma, pL, rhoL, pR, rhoR):
    """Right-going shock speed of the perfect-gas Riemann problem with uL = uR = 0."""
    cL, cR = np.sqrt(gamma * pL / rhoL), np.sqrt(gamma * pR / rhoR)

    def f(p, pk, rk, ck):
        if p > pk:   # shock branch
            A, B = 2.0 / ((gamma + 1) * rk), (gamma - 1) / (gamma + 1) * pk
            q = np.sqrt(A / (p + B))
            return (p - pk) * q, q * (1 - 0.5 * (p - pk) / (p + B))
        pr = p / pk  # rarefaction branch
        return 2 * ck / (gamma - 1) * (pr ** ((gamma - 1) / (2 * gamma)) - 1), \
            1.0 / (rk * ck) * pr ** (-(gamma + 1) / (2 * gamma))

    p = 0.5 * (pL + pR)
    for _ in range(100):
        fL, dL = f(p, pL, rhoL, cL)
        fR, dR = f(p, pR, rhoR, cR)
        dp = (fL + fR) / (dL + dR)
        p -= dp
        if abs(dp) < 1e-13 * p:
            break
    S = cR * np.sqrt((gamma + 1) / (2 * gamma) * p / pR + (gamma - 1) / (2 * gamma))
    return S, p


def test_shock_speed_matches_exact_riemann_solution():
    n = 800
    mech, tube = _riemann_tube(n)
    rho, u, T, p, Y = tube.primitives()
    _, cp = tube.th.h_cp(np.array([300.0]))
    cpm = float((Y[:, -1:] * cp).sum())
    rmix = float(flow1d.RU * (Y[:, -1] / tube.th.W).sum())
    gamma = cpm / (cpm - rmix)
    S, pstar = _exact_shock_speed(gamma, p[0], rho[0], p[-1], rho[-1])
    dt = 0.3 * tube.dx / tube.max_wave_speed()
    steps = int(0.35 / (S * dt))
    for _ in range(steps):
        tube.step(dt)
    _, _, _, p1, _ = tube.primitives()
    x = (np.arange(n) + 0.5) / n
    mid = 0.5 * (pstar + p[-1])
    right = x > 0.5
    idx = np.where(right & (p1 < mid))[0][0]          # first cell right of the diaphragm below the mean
    x_num = x[idx - 1] + (p1[idx - 1] - mid) / (p1[idx - 1] - p1[idx]) * (x[idx] - x[idx - 1])
    x_ex = 0.5 + S * steps * dt
    assert abs(x_num - x_ex) <= max(3 * tube.dx, 0.01 * (x_ex - 0.5)), (x_num, x_ex, tube.dx)
