"""The batched 54 x 54 LU of the large-mechanism comparison, both trailing-update
paths (FP64 tensor cores and CUDA cores), against LAPACK's getrf (scipy).

Matrices are shaped like the large-mechanism systems I/(gamma h) - J: a dominant
diagonal plus seeded off-diagonal entries spanning several orders of magnitude,
and a set of plain random matrices whose pivoting is non-trivial.  Pivots must
equal LAPACK's exactly (no ties in continuous random data); the factors agree to
rounding (1e-12 relative to the largest entry of the row of U / column of L)."""
import numpy as np
import pytest
import torch

from gpu_util import library
from paper_2508_16105_gb300 import rde_chem, synth

pytestmark = pytest.mark.gpu
scipy_linalg = pytest.importorskip("scipy.linalg")


def matrices(batch, n, seed):
    r = synth.normal(seed, "lu", batch * n * n).reshape(batch, n, n)
    A = r.copy()
    A[: batch // 2] *= np.exp(2.0 * synth.normal(seed + 1, "scale", (batch // 2) * n * n)).reshape(batch // 2, n, n)
    idx = np.arange(n)
    A[: batch // 2, idx, idx] += 50.0      # M = I/(gamma h) - J: a dominant diagonal
    return A


@pytest.mark.parametrize("n", [54, 7, 56, 1])
@pytest.mark.parametrize("dmma", [0, 1])
def test_batched_lu_matches_lapack(n, dmma):
    library()
    batch = 97
    A = matrices(batch, n, 31 + n)
    d = torch.tensor(A, device="cuda")
    piv = torch.zeros((batch, n), dtype=torch.int32, device="cuda")
    info = torch.full((batch,), -1, dtype=torch.int32, device="cuda")
    rde_chem.rde_selftest_batched_lu(dmma, d, piv, info)
    torch.cuda.synchronize()
    LU, P, I = d.cpu().numpy(), piv.cpu().numpy(), info.cpu().numpy()
    assert (I == 0).all()
    for b in range(batch):
        lu, pv = scipy_linalg.lu_factor(A[b])
        assert np.array_equal(P[b], pv), b
        scale = np.maximum(np.abs(lu).max(axis=1, keepdims=True), np.abs(lu).max(axis=0, keepdims=True))
        assert (np.abs(LU[b] - lu) <= 1e-12 * scale).all(), (b, np.abs(LU[b] - lu).max())


def test_singular_and_zero_batch():
    library()
    A = np.eye(9)[None].repeat(3, axis=0)
    A[1, 4, 4] = 0.0
    A[1, 4, :] = 0.0           # row 4 all zero: the fifth pivot is zero
    d = torch.tensor(A, device="cuda")
    piv = torch.zeros((3, 9), dtype=torch.int32, device="cuda")
    info = torch.zeros(3, dtype=torch.int32, device="cuda")
    for dmma in (0, 1):
        rde_chem.rde_selftest_batched_lu(dmma, d.clone(), piv, info)
        torch.cuda.synchronize()
        assert info.cpu().tolist() == [0, 5, 0]
    e = torch.zeros((0, 5, 5), dtype=torch.float64, device="cuda")
    rde_chem.rde_selftest_batched_lu(1, e, torch.zeros((0, 5), dtype=torch.int32, device="cuda"))
    with pytest.raises(rde_chem.RdeError):
        rde_chem.rde_selftest_batched_lu(0, torch.zeros((2, 57, 57), dtype=torch.float64, device="cuda"),
                                         torch.zeros((2, 57), dtype=torch.int32, device="cuda"))
