"""The Python binding refuses cell blocks whose (n, ldY) reach beyond their tensors'
storage: the kernels index Y[k * ldY + i] and the per-cell vectors up to n without
any bound they could check, so the binding checks them on the host (CPU tensors
suffice: only shapes, strides and storage sizes are read)."""
import pytest
import torch

from paper_2508_16105_gb300 import rde_chem


def _cells(K=9, n=10, ld=None):
    ld = n if ld is None else ld
    return torch.zeros(n, dtype=torch.float64), torch.zeros(n, dtype=torch.float64), \
        torch.zeros(K, ld, dtype=torch.float64)


def test_consistent_blocks_pass():
    p, T, Y = _cells()
    b = rde_chem.make_block(p, T, Y)
    assert b.n == 10 and b.ldY == 10
    # padded leading dimension and a suffix view (its storage runs to the end)
    p, T, Y = _cells(n=10, ld=13)
    assert rde_chem.make_block(p, T, Y).ldY == 13
    assert rde_chem.make_block(p[4:], T[4:], Y[:, 4:], n=6, ldY=13).n == 6
    # a one-cell copy is its own species-major array with ldY 1
    assert rde_chem.make_block(p[:1], T[:1].clone(), Y[:, :1].clone()).ldY == 1
    # empty blocks are not checked
    assert rde_chem.make_block(p[:0], T[:0], Y[:, :0], n=0, ldY=0).n == 0


def test_out_of_storage_blocks_raise():
    p, T, Y = _cells()
    with pytest.raises(ValueError):   # a one-cell copy of Y given the field's ldY
        rde_chem.make_block(p[:1], T[:1], Y[:, :1].clone(), n=1, ldY=10)
    with pytest.raises(ValueError):   # more cells than T's storage holds
        rde_chem.make_block(p, torch.zeros(5, dtype=torch.float64), Y, n=10, ldY=10)
    with pytest.raises(ValueError):   # ldY below the cell count
        rde_chem.make_block(p, T, Y, n=10, ldY=9)
    with pytest.raises(ValueError):   # cell-major Y
        rde_chem.make_block(p, T, torch.zeros(10, 9, dtype=torch.float64).t())
    with pytest.raises(ValueError):   # an output vector shorter than n
        rde_chem.make_block(p, T, Y, status=torch.zeros(3, dtype=torch.int32))
