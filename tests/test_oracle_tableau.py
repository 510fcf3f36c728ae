"""Pins for the Rosenbrock coefficients (RODAS3, Sandu et al. 1997).

The oracle stores the method in the transformed form (gamma, a_ij, c_ij, m_i,
e_i).  Converting back to the classical parameters (alpha_ij, gamma_ij, b_i) of
Hairer & Wanner, Solving ODEs II, Section IV.7, the order conditions of
their Table 7.1 must hold through order 3 for the main method and order 2 for
the embedded one; the method must be L-stable (R(inf) = 0) and A-stable on the
imaginary axis.  A mistyped coefficient breaks one of these.
"""
import numpy as np
import pytest

import oracle


def classical():
    g, a, c, m, e = oracle.tableau()
    s = 4
    Ginv = np.diag(np.full(s, 1.0 / g)) - np.tril(c, -1)
    G = np.linalg.inv(Ginv)
    alpha = np.tril(a, -1) @ G
    b = m @ G
    bhat = (m - e) @ G
    return g, alpha, G, b, bhat


def test_gamma_diagonal():
    g, alpha, G, b, bhat = classical()
    assert np.allclose(np.diag(G), g)
    assert np.allclose(np.triu(alpha), 0.0)


def conditions(b, alpha, G, g):
    beta = np.tril(alpha + G, -1)
    a_i = alpha.sum(1)
    b_i = beta.sum(1)
    return {
        1: [(b.sum(), 1.0)],
        2: [(b @ b_i, 0.5 - g)],
        3: [(b @ a_i ** 2, 1.0 / 3.0), (b @ (beta @ b_i), 1.0 / 6.0 - g + g * g)],
    }


def test_order3_main():
    g, alpha, G, b, bhat = classical()
    for order, conds in conditions(b, alpha, G, g).items():
        for lhs, rhs in conds:
            assert abs(lhs - rhs) < 1e-14, (order, lhs, rhs)


def test_order2_embedded_and_not_3():
    g, alpha, G, b, bhat = classical()
    c = conditions(bhat, alpha, G, g)
    for order in (1, 2):
        for lhs, rhs in c[order]:
            assert abs(lhs - rhs) < 1e-14
    # the embedded method must differ from the main one (else the estimate is zero)
    assert max(abs(l - r) for l, r in c[3]) > 1e-3


def stability(z, b, alpha, G):
    B = alpha + G
    s = len(b)
    return 1.0 + z * b @ np.linalg.solve(np.eye(s) - z * B, np.ones(s))


def test_L_stable():
    g, alpha, G, b, bhat = classical()
    B = alpha + G
    R_inf = 1.0 - b @ np.linalg.solve(B, np.ones(4))
    assert abs(R_inf) < 1e-14
    assert abs(stability(-1e12, b, alpha, G)) < 1e-10


@pytest.mark.parametrize("y", np.concatenate([np.logspace(-3, 4, 40), -np.logspace(-3, 4, 40)]))
def test_A_stable_imag_axis(y):
    g, alpha, G, b, bhat = classical()
    assert abs(stability(1j * y, b, alpha, G)) <= 1.0 + 1e-12


def test_stability_matches_exp_for_small_z():
    g, alpha, G, b, bhat = classical()
    for z in (1e-2, -1e-2, 2e-2j):
        # order 3: R(z) - e^z = O(z^4)
        assert abs(stability(z, b, alpha, G) - np.exp(z)) < 5 * abs(z) ** 4
