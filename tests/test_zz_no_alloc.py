"""The allocation-free entry point, rde_chem_advance_noalloc.

Some callers cannot allocate device memory while they advance the chemistry:
code recording a CUDA graph, latency-critical loops that forbid allocator
calls, and applications whose device memory belongs to another allocator.  For
them the library keeps the queue kernel's small scratch (work-queue counter and
statistics) in a static device array instead of the per-handle buffer.  This
test calls that entry point through the C ABI twice in a row and checks that
each call reproduces rde_chem_advance_ex on the same cells.  The file is named
so that pytest collects it last.
"""
import numpy as np
import pytest
import torch

from gpu_util import T_REL_TOL, Y_ABS_TOL, library, to_dev
from paper_2508_16105_gb300 import rde_chem, synth

pytestmark = pytest.mark.gpu


def _run(entry, m, cells, dt):
    n = cells.n
    p, T, Y = to_dev(cells.p), to_dev(cells.T), to_dev(cells.Y)
    st = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    na = torch.zeros(n, dtype=torch.int32, device="cuda")
    blk = rde_chem.make_block(p, T, Y, status=st, n_acc=na, n=n, ldY=n)
    entry(m.handle, dt, cells=blk)
    torch.cuda.synchronize()
    return T.cpu().numpy(), Y.cpu().numpy(), st.cpu().numpy(), na.cpu().numpy()


def test_noalloc_matches_advance_ex_twice():
    library()
    mech = synth.h2_air_mechanism(16105)
    cells = synth.field_cells(mech, 3000, seed=1002)
    m = rde_chem.Mechanism(mech.to_text())
    T0, Y0, s0, a0 = _run(rde_chem.rde_chem_advance_ex, m, cells, 5e-9)
    assert (s0 == 0).all()
    for _ in range(2):
        T1, Y1, s1, a1 = _run(rde_chem.rde_chem_advance_noalloc, m, cells, 5e-9)
        assert np.array_equal(s1, s0)
        assert np.array_equal(a1, a0)
        assert (np.abs(T1 - T0) / T0).max() <= T_REL_TOL
        assert np.abs(Y1 - Y0).max() <= Y_ABS_TOL
    m.close()
