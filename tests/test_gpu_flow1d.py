"""The chemistry step inside an operator-split 1D reacting flow: a closed tube of
burnt, post-shock and fresh H2-air regions (the seeded 9-species mechanism),
advanced for 12 split steps (transport, then the chemistry of every cell over the
same dt with its step-size hint carried).  The run with the sm_103a library as the
chemistry operator matches the same split with the CPU oracle as the chemistry
operator: |dT|/T <= 1e-6 and |dY_k| <= 1e-8 after the 12 steps (the one-step
chemistry bounds, Y widened tenfold for the 12 coupled steps)."""
import os

import numpy as np
import pytest

import oracle
from gpu_util import library
from paper_2508_16105_gb300 import flow1d, rde_chem, synth

pytestmark = pytest.mark.gpu


def _tube(mech, n=96):
    cells = synth.field_cells(mech, 4000, seed=1002)
    pick = {c: int(np.where(cells.cls == c)[0][0]) for c in (0, 1, 2)}
    x = (np.arange(n) + 0.5) / n
    region = np.where(x < 0.3, 2, np.where(x < 0.45, 1, 0))      # burnt | front | fresh
    T = np.array([{2: 2200.0, 1: 1800.0, 0: 600.0}[r] for r in region])
    p = np.array([{2: 1.0e6, 1: 1.5e6, 0: 2.0e5}[r] for r in region])
    Y = np.stack([cells.Y[:, pick[r]] for r in region], axis=1)
    return flow1d.Tube(mech, p, T, Y, length=2e-3)


def test_split_flow_gpu_chemistry_matches_oracle_chemistry():
    library()
    mech = synth.h2_air_mechanism(16105)
    m = rde_chem.Mechanism(mech.to_text())
    o = oracle.Oracle(mech.to_text())

    def oracle_chem(p, T, Y, dt, hint):
        T2, Y2, st, _, _, h2 = o.advance(p, T, Y, dt, hint=hint, threads=os.cpu_count())
        assert (st == 0).all()
        return T2, Y2, h2

    a, b = _tube(mech), _tube(mech)
    dt = 0.4 * a.dx / a.max_wave_speed()
    gpu = flow1d.library_chemistry(m.handle)
    for _ in range(12):
        a.step(dt, gpu)
        b.step(dt, oracle_chem)
    m.close()
    _, _, Ta, pa, Ya = a.primitives()
    _, _, Tb, pb, Yb = b.primitives()
    assert np.abs(Ta - Tb).max() / Tb.min() <= 1e-6, np.abs(Ta - Tb).max()
    assert np.abs(Ya - Yb).max() <= 1e-8, np.abs(Ya - Yb).max()
    # the chemistry did something: the front region heated or cooled by more than the bound
    c = _tube(mech)
    for _ in range(12):
        c.step(dt)
    _, _, Tc, _, _ = c.primitives()
    assert np.abs(Ta - Tc).max() > 1.0
