"""The oracle's dense LU with partial pivoting against numpy.linalg.solve."""
import numpy as np

import oracle
from paper_2508_16105_gb300 import synth


def test_random_systems():
    for n in (2, 3, 10, 54):
        u = synth.uniform(5, "lu/%d" % n, n * n + 3 * n)
        A = (u[:n * n].reshape(n, n) - 0.5) + np.diag(np.full(n, 0.1))
        B = u[n * n:].reshape(3, n)
        rc, X = oracle.lu_solve(A, B)
        assert rc == 0
        ref = np.linalg.solve(A, B.T).T
        assert np.abs(X - ref).max() < 1e-10 * np.abs(ref).max()


def test_needs_pivoting():
    A = np.array([[0.0, 2.0, 1.0], [1.0, 1.0, 0.0], [3.0, 0.0, 1.0]])
    b = np.array([[1.0, 2.0, 3.0]])
    rc, x = oracle.lu_solve(A, b)
    assert rc == 0
    assert np.allclose(A @ x[0], b[0], rtol=0, atol=1e-14)


def test_singular():
    A = np.array([[1.0, 2.0], [2.0, 4.0]])
    A[1] = 2 * A[0]
    A2 = np.array([[0.0, 1.0], [0.0, 3.0]])
    rc, _ = oracle.lu_solve(A2, np.array([[1.0, 1.0]]))
    assert rc == -1
