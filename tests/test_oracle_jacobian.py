"""The oracle's analytic Jacobian against central finite differences of its RHS.

Central differences with relative step 1e-3 and 5e-4 per variable, combined by
Richardson extrapolation (truncation O(h^4)); the difference is measured
row-wise against the largest entry of the row.
"""
import numpy as np
import pytest

import oracle
from paper_2508_16105_gb300 import synth


def central(o, p, y, rel):
    N = len(y)
    J = np.zeros((N, N))
    for j in range(N):
        h = rel * abs(y[j]) if y[j] != 0 else rel * 1e-3
        yp, ym = y.copy(), y.copy()
        yp[j] += h
        ym[j] -= h
        J[:, j] = (o.rhs(p, yp) - o.rhs(p, ym)) / (yp[j] - ym[j])
    return J


def fd_jac(o, p, y, rel=1e-3):
    return (4.0 * central(o, p, y, rel / 2) - central(o, p, y, rel)) / 3.0


def check(o, p, y, tol):
    f, J = o.jac(p, y)
    Jfd = fd_jac(o, p, y)
    scale = np.abs(Jfd).max(axis=1, keepdims=True) + 1e-300
    err = (np.abs(J - Jfd) / scale).max()
    assert err < tol, err
    assert np.allclose(f, o.rhs(p, y), rtol=0, atol=0)


def test_jacobian_h2(h2mech, h2oracle):
    cells = synth.uniform_cells(h2mech, 200, seed=11)
    for i in range(cells.n):
        check(h2oracle, cells.p[i], np.append(cells.Y[:, i], cells.T[i]), 1e-7)


def test_jacobian_field_classes(h2mech, h2oracle):
    cells = synth.field_cells(h2mech, 300, seed=12)
    for i in range(cells.n):
        check(h2oracle, cells.p[i], np.append(cells.Y[:, i], cells.T[i]), 1e-7)


@pytest.mark.parametrize("troe", [(0.6, 150.0, 2500.0), (0.4, 300.0, 1800.0, 5000.0)])
def test_jacobian_falloff(troe):
    # a falloff reaction with a genuinely T- and M-dependent blending, plus an inert
    mech = synth.isomer_mechanism(kind="TROE", reversible=True, A=3.0e5, b=0.3, E=40.0,
                                  low=(4.0e12, -0.5, 10.0), troe=troe)
    mech.reactions[0].eff = {"X2": 2.0, "A": 0.7}
    o = oracle.Oracle(mech.to_text())
    for T in (700.0, 1300.0, 2200.0):
        for p in (2e4, 1e5, 2e6):
            check(o, p, np.array([0.5, 0.2, 0.3, T]), 1e-7)


def test_jacobian_two_range():
    mech = synth.two_range_mechanism()
    o = oracle.Oracle(mech.to_text())
    for T in (600.0, 999.0, 1001.0, 1700.0):
        check(o, 1e5, np.array([0.7, 0.3, T]), 1e-7)
