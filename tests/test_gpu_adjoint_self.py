"""The self-contained adjoint (rde_chem_advance_adjoint: no step counts from the caller).

The caller advances the cells with the plain rde_chem_advance (no n_acc array) and
then asks for the gradient with only the step's inputs, dt, the cotangents and a
workspace sized by rde_chem_adjoint_workspace(h, n, dt).  The library keeps S
checkpoints per cell, thinned by powers of two, and replays segments from them when
a cell took more than S steps.  Checks:
  - per-cell state gradients and the adjoint identity against the oracle's exact
    (complex-step) tangent of the same frozen step sequence, 1e-7 of the size of
    the terms (the bound of the recorded adjoint's test);
  - the self-checkpointing gradients equal those of the recorded mode (the caller's
    n_acc) to 1e-12, with the default S and with S = 64 (every cell replays);
  - the CTA-per-cell adjoint in the same mode (replays included) against its
    recorded mode.
"""
import numpy as np
import pytest
import torch

import oracle
from gpu_util import library, to_dev
from paper_2508_16105_gb300 import rde_chem, synth

pytestmark = pytest.mark.gpu


def _cot(seed, K, n):
    g = synth.normal(seed, "cot", (K + 1) * n).reshape(K + 1, n)
    return g[K].copy(), g[:K].copy()


def _outs(m, n):
    return (torch.empty(n, dtype=torch.float64, device="cuda"), torch.empty((m.K, n), dtype=torch.float64, device="cuda"),
            torch.empty(m.R, dtype=torch.float64, device="cuda"), torch.empty(m.R, dtype=torch.float64, device="cuda"))


def _self(m, dt, p, T0, Y0, gT, gY, nbytes=None, block=False):
    n = int(T0.shape[0])
    gT0, gY0, glnA, gE = _outs(m, n)
    if nbytes is None:
        nbytes = rde_chem.rde_chem_adjoint_workspace(m.handle, n, dt)
    ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    st = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    if block:
        rde_chem.rde_chem_advance_adjoint_ex(m.handle, dt, p, T0, Y0, None, 0, gT, gY, gT0, gY0, glnA, gE, ws,
                                             status=st, schedule=rde_chem.RDE_SCHED_BLOCK)
    else:
        rde_chem.rde_chem_advance_adjoint_ex(m.handle, dt, p, T0, Y0, None, 0, gT, gY, gT0, gY0, glnA, gE, ws,
                                             status=st)
    torch.cuda.synchronize()
    return dict(gT0=gT0.cpu().numpy(), gY0=gY0.cpu().numpy(), glnA=glnA.cpu().numpy(), gE=gE.cpu().numpy(),
                status=st.cpu().numpy())


def _recorded(m, dt, p, T0, Y0, gT, gY, block=False):
    n = int(T0.shape[0])
    T, Y = T0.clone(), Y0.clone()
    n_acc = torch.zeros(n, dtype=torch.int32, device="cuda")
    sched = rde_chem.RDE_SCHED_BLOCK if block else rde_chem.RDE_SCHED_AUTO
    rde_chem.rde_chem_advance_ex(m.handle, dt, cells=rde_chem.make_block(p, T, Y, n_acc=n_acc), schedule=sched,
                                 threads_per_cta=128)
    total = int(n_acc.sum().item())
    ws = torch.empty(rde_chem.rde_chem_adjoint_workspace_steps(m.handle, n, total), dtype=torch.uint8, device="cuda")
    gT0, gY0, glnA, gE = _outs(m, n)
    st = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    rde_chem.rde_chem_advance_adjoint_ex(m.handle, dt, p, T0, Y0, n_acc, total, gT, gY, gT0, gY0, glnA, gE, ws,
                                         status=st, schedule=sched)
    torch.cuda.synchronize()
    return dict(gT0=gT0.cpu().numpy(), gY0=gY0.cpu().numpy(), glnA=glnA.cpu().numpy(), gE=gE.cpu().numpy(),
                status=st.cpu().numpy(), n_acc=n_acc.cpu().numpy())


def _close(a, b, rel):
    for k in ("gT0", "gY0", "glnA", "gE"):
        scale = max(np.abs(b[k]).max(), 1e-300)
        assert np.abs(a[k] - b[k]).max() <= rel * scale, (k, np.abs(a[k] - b[k]).max(), scale)


def test_flat_call_after_plain_advance_matches_oracle_tangent(h2mech):
    """rde_chem_advance, then the flat self-contained call: no n_acc anywhere."""
    library()
    cells = synth.uniform_cells(h2mech, 16, seed=1001)
    n, dt, N = cells.n, 1e-8, h2mech.K + 1
    m = rde_chem.Mechanism(h2mech.to_text())
    p, T0, Y0 = to_dev(cells.p), to_dev(cells.T), to_dev(cells.Y)
    T, Y = T0.clone(), Y0.clone()
    rde_chem.rde_chem_advance(m.handle, n, p, T, Y, dt)
    gT_h, gY_h = _cot(2011, h2mech.K, n)
    gT, gY = to_dev(gT_h), to_dev(gY_h)
    gT0, gY0, glnA, gE = _outs(m, n)
    ws = torch.empty(rde_chem.rde_chem_adjoint_workspace(m.handle, n, dt), dtype=torch.uint8, device="cuda")
    rde_chem.rde_chem_advance_adjoint(m.handle, dt, p, T0, Y0, gT, gY, gT0, gY0, glnA, gE, ws)
    torch.cuda.synchronize()
    g_T0, g_Y0 = gT0.cpu().numpy(), gY0.cpu().numpy()
    g_lnA, g_E = glnA.cpu().numpy(), gE.cpu().numpy()
    # the GPU's step counts, only to pick the cells whose oracle sequence has the same length
    na = torch.zeros(n, dtype=torch.int32, device="cuda")
    Tc, Yc = T0.clone(), Y0.clone()
    rde_chem.rde_chem_advance_ex(m.handle, dt, cells=rde_chem.make_block(p, Tc, Yc, n_acc=na), threads_per_cta=128)
    n_acc = na.cpu().numpy()
    m.close()
    o = oracle.Oracle(h2mech.to_text())
    R = h2mech.R
    dlnA = synth.uniform(5, "dlnA", R) - 0.5
    dE = (synth.uniform(5, "dE", R) - 0.5) * 1e3
    lhs = rhs = 0.0
    same = 0
    for i in range(n):
        y0 = np.append(cells.Y[:, i], cells.T[i])
        rc, _, steps = oracle.record(o, cells.p[i], y0, dt)
        if len(steps) != n_acc[i]:
            continue
        same += 1
        gbar = np.append(gY_h[:, i], gT_h[i])
        for j in range(N):
            e = np.zeros(N)
            e[j] = 1.0
            _, tj = oracle.tangent(o, cells.p[i], y0, steps, dy0=e)
            gj = g_Y0[j, i] if j < N - 1 else g_T0[i]
            mag = np.abs(gbar * tj).sum()
            assert abs(gbar @ tj - gj) <= 1e-7 * mag + 1e-300, (i, j, gbar @ tj, gj)
        dy0 = (synth.uniform(6 + i, "dy0", N) - 0.5) * np.append(np.full(N - 1, 1e-3), 10.0)
        _, t = oracle.tangent(o, cells.p[i], y0, steps, dy0=dy0, dlnA=dlnA, dE=dE)
        lhs += gbar @ t
        rhs += np.append(g_Y0[:, i], g_T0[i]) @ dy0
    assert same >= n - 2
    if same == n:
        rhs += g_lnA @ dlnA + g_E @ dE
        assert abs(lhs - rhs) <= 1e-7 * max(abs(lhs), 1e-300), (lhs, rhs)


@pytest.mark.parametrize("S", [None, 64])
def test_self_checkpointing_matches_recorded(h2mech, S):
    """Default S (cells of a few hundred steps fit) and S = 64 (every cell replays
    segments from thinned checkpoints): both equal the recorded mode's gradients."""
    library()
    cells = synth.field_cells(h2mech, 600, seed=1004, fractions=(0.25, 0.50, 0.25))
    n, dt = cells.n, 1e-8
    m = rde_chem.Mechanism(h2mech.to_text())
    p, T0, Y0 = to_dev(cells.p), to_dev(cells.T), to_dev(cells.Y)
    gT_h, gY_h = _cot(2012, h2mech.K, n)
    gT, gY = to_dev(gT_h), to_dev(gY_h)
    rec = _recorded(m, dt, p, T0, Y0, gT, gY)
    assert (rec["status"] == 0).all()
    nbytes = None if S is None else rde_chem.rde_selftest_adjoint_self_workspace(m.handle, n, S)
    if S is not None:
        assert rec["n_acc"].min() > S        # every cell replays segments
    slf = _self(m, dt, p, T0, Y0, gT, gY, nbytes)
    m.close()
    assert (slf["status"] == 0).all(), np.bincount(slf["status"])
    _close(slf, rec, 1e-12)


def test_self_checkpointing_workspace_bounds(h2mech):
    """The query covers the default layout; a workspace below every layout (S = 16 ..
    1024 checkpoints; the replay segment grows as S shrinks) is refused on the host."""
    library()
    m = rde_chem.Mechanism(h2mech.to_text())
    n = 1000
    full = rde_chem.rde_chem_adjoint_workspace(m.handle, n, 1e-8)
    sizes = [rde_chem.rde_selftest_adjoint_self_workspace(m.handle, n, 1 << e) for e in range(4, 11)]
    assert all(x > 0 for x in sizes) and full >= min(sizes[-2:])
    small = min(sizes)
    assert rde_chem.rde_chem_adjoint_workspace(m.handle, n, 0.0) == 0
    assert rde_chem.rde_chem_adjoint_workspace(m.handle, -1, 1e-8) == 0
    # a workspace below the smallest layout is refused before any launch
    z = torch.zeros(n, dtype=torch.float64, device="cuda")
    zy = torch.zeros((m.K, n), dtype=torch.float64, device="cuda")
    gT0, gY0, glnA, gE = _outs(m, n)
    ws = torch.empty(small - 256, dtype=torch.uint8, device="cuda")
    with pytest.raises(rde_chem.RdeError) as ei:
        rde_chem.rde_chem_advance_adjoint(m.handle, 1e-8, z + 1e5, z + 1000.0, zy, z, zy, gT0, gY0, glnA, gE, ws)
    assert ei.value.code == -8
    m.close()


def test_block_adjoint_self_checkpointing_with_replays():
    """The CTA-per-cell adjoint without step counts, with 16 checkpoints per CTA so
    that its cells replay segments, equals its recorded mode."""
    library()
    mech = synth.h2_air_mechanism(16105)
    cells = synth.field_cells(mech, 48, seed=1004, fractions=(0.25, 0.50, 0.25))
    n, dt = cells.n, 1e-8
    m = rde_chem.Mechanism(mech.to_text())
    p, T0, Y0 = to_dev(cells.p), to_dev(cells.T), to_dev(cells.Y)
    gT_h, gY_h = _cot(2013, mech.K, n)
    gT, gY = to_dev(gT_h), to_dev(gY_h)
    rec = _recorded(m, dt, p, T0, Y0, gT, gY, block=True)
    assert (rec["status"] == 0).all() and rec["n_acc"].min() > 16
    nbytes = rde_chem.rde_selftest_adjoint_self_workspace(m.handle, n, 16, block=True)
    slf = _self(m, dt, p, T0, Y0, gT, gY, nbytes, block=True)
    m.close()
    assert (slf["status"] == 0).all(), np.bincount(slf["status"])
    _close(slf, rec, 1e-12)
