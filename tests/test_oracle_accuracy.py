"""Accuracy of the oracle's integrator.

- Fixed-step convergence on the nonlinear dimerisation 2A -> B (closed form
  1/Y - ln Y = 1/Y0 - ln Y0 + kappa t): the global error falls as h^3, and the
  embedded error estimate (the order-2 companion) as h^3 per step.
- Adaptive runs at rtol 1e-8 / atol 1e-12 on the 9-species mechanism against
  scipy's Radau IIA at rtol 1e-12 on the same right-hand side: the integrator's
  own global error is far inside the parity tolerances |dT|/T <= 1e-6 and
  |dY| <= 1e-9.  On 3 uniform cells, and on 32 cells of the workloads' four
  classes (8 uniform at dt 1e-8; 8 fresh, 8 post-shock front and 8 burnt cells of
  the RDE-like field at dt 5e-9).
- The error distribution over 256 such cells (64 per class): the run at rtol
  1e-8 against the same integrator at rtol 1e-12 / atol 1e-16 (its converged
  answer, itself within 1e-12 of Radau on the cells above).
"""
import numpy as np
from scipy.integrate import solve_ivp

import oracle
from paper_2508_16105_gb300 import synth

RU = 8.31446261815324


def dimer_exact(Y0, kappa, t):
    rhs = 1 / Y0 - np.log(Y0) + kappa * t
    y = Y0
    for _ in range(80):
        y -= (1 / y - np.log(y) - rhs) / (-1 / y ** 2 - 1 / y)
    return y


def test_fixed_step_order3():
    A, b, E, T, p = 3.0e9, 0.0, 0.0, 900.0, 2.0e5
    mech = synth.dimer_mechanism(A=A, b=b, E=E)
    o = oracle.Oracle(mech.to_text())
    k = A * 1e-6
    kappa = 4 * k * p / (RU * T)
    t_end = 2.0 / kappa
    errs, ests = [], []
    for n in (10, 20, 40, 80):
        h = t_end / n
        y = np.array([0.9, 0.1, T])
        for i in range(n):
            rc, y, e = o.fixed_step(p, y, h)
            if i == 0:
                ests.append(abs(e[0]))
        errs.append(abs(y[0] - dimer_exact(0.9, kappa, t_end)))
    slopes = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert (slopes > 2.7).all() and (slopes < 3.4).all(), slopes
    est_slopes = np.log2(np.array(ests[:-1]) / np.array(ests[1:]))
    assert (est_slopes > 2.7).all(), est_slopes


def test_adaptive_vs_radau(h2mech, h2oracle):
    cells = synth.uniform_cells(h2mech, 3, seed=1001)
    T, Y, st, na, nr, _ = h2oracle.advance(cells.p, cells.T, cells.Y, 1e-8)
    assert (st == 0).all()
    for i in range(cells.n):
        p = cells.p[i]
        y0 = np.append(cells.Y[:, i], cells.T[i])
        sol = solve_ivp(lambda t, y: h2oracle.rhs(p, y), (0, 1e-8), y0, method="Radau",
                        rtol=1e-12, atol=1e-18, jac=lambda t, y: h2oracle.jac(p, y)[1])
        ref = sol.y[:, -1]
        assert abs(T[i] - ref[-1]) / ref[-1] < 1e-7
        assert np.abs(Y[:, i] - ref[:-1]).max() < 2e-10


def _class_cells(mech, per_class):
    """per_class uniform cells (dt 1e-8) and per_class cells of each field class (dt 5e-9)."""
    out = [("uniform", synth.uniform_cells(mech, per_class, seed=1001), 1e-8)]
    field = synth.field_cells(mech, 40 * per_class, seed=1002)
    for c, name in ((0, "fresh"), (1, "front"), (2, "burnt")):
        idx = np.where(field.cls == c)[0][:per_class]
        assert len(idx) == per_class
        out.append((name, synth.subset(field, idx), 5e-9))
    return out


def test_adaptive_vs_radau_all_classes(h2mech, h2oracle):
    for name, cells, dt in _class_cells(h2mech, 8):
        T, Y, st, _, _, _ = h2oracle.advance(cells.p, cells.T, cells.Y, dt)
        assert (st == 0).all(), name
        for i in range(cells.n):
            p = cells.p[i]
            y0 = np.append(cells.Y[:, i], cells.T[i])
            sol = solve_ivp(lambda t, y: h2oracle.rhs(p, y), (0, dt), y0, method="Radau",
                            rtol=1e-12, atol=1e-18, jac=lambda t, y: h2oracle.jac(p, y)[1])
            ref = sol.y[:, -1]
            assert abs(T[i] - ref[-1]) / ref[-1] < 1e-7, (name, i)
            assert np.abs(Y[:, i] - ref[:-1]).max() < 2e-10, (name, i)


def test_error_distribution_256_cells(h2mech, h2oracle):
    import os
    tight = oracle.default_opts(rtol=1e-12, atol=1e-16)
    report = {}
    for name, cells, dt in _class_cells(h2mech, 64):
        T, Y, st, _, _, _ = h2oracle.advance(cells.p, cells.T, cells.Y, dt, threads=os.cpu_count())
        Tr, Yr, sr, _, _, _ = h2oracle.advance(cells.p, cells.T, cells.Y, dt, tight, threads=os.cpu_count())
        assert (st == 0).all() and (sr == 0).all(), name
        dT = np.abs(T - Tr) / Tr
        dY = np.abs(Y - Yr).max(axis=0)
        report[name] = (np.percentile(dT, [50, 90, 100]), np.percentile(dY, [50, 90, 100]))
        assert dT.max() < 1e-7 and dY.max() < 2e-10, (name, dT.max(), dY.max())
    for name, (t, y) in report.items():
        print("%-8s |dT|/T p50 %.1e p90 %.1e max %.1e   max_k |dY_k| p50 %.1e p90 %.1e max %.1e"
              % (name, t[0], t[1], t[2], y[0], y[1], y[2]))

