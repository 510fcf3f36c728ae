"""The discrete adjoint on the GPU against the oracle's exact tangent.

For cells whose GPU and oracle integrations take the same number of accepted
steps (the same frozen map), the adjoint identity
    sum_cells <gbar, TLM_cell (dy0_cell, dlnA, dE)> = sum_cells <gy0_cell, dy0_cell> + <g_lnA, dlnA> + <g_E, dE>
must hold (the oracle's TLM is a complex-step derivative of its own frozen-step
replay), and per-cell state gradients must match the oracle tangent component
by component.  The two sides differ only by rounding along trajectories of
~700 steps (a rounding-level difference in the states moves the products of
the step Jacobians by ~1e-8 relative), so the bound is 1e-7 of the size of the
terms; an omitted or mis-signed adjoint term is orders of magnitude larger.  The
parameter gradients must match the oracle's complex-step tangent and central
finite differences of the frozen replay (h = 1e-4 relative).  Also: determinism, autograd wiring, and falloff /
efficiency code paths on small mechanisms.
"""
import numpy as np
import pytest
import torch

import oracle
from gpu_util import library, small_case, to_dev
from paper_2508_16105_gb300 import autograd, rde_chem, synth

pytestmark = pytest.mark.gpu


def gpu_adjoint(mech, cells, dt, gT, gY, rtol=1e-8, atol=1e-12, stages=False, total_steps=None):
    library()
    m = rde_chem.Mechanism(mech.to_text(), rtol, atol)
    n = cells.n
    p, T0, Y0 = to_dev(cells.p), to_dev(cells.T), to_dev(cells.Y)
    T, Y = T0.clone(), Y0.clone()
    n_acc = torch.zeros(n, dtype=torch.int32, device="cuda")
    rde_chem.rde_chem_advance_ex(m.handle, dt, cells=rde_chem.make_block(p, T, Y, n_acc=n_acc), threads_per_cta=128)
    total = int(n_acc.sum().item()) if total_steps is None else total_steps
    size = (rde_chem.rde_chem_adjoint_workspace_checkpointed if stages else rde_chem.rde_chem_adjoint_workspace_steps)(
        m.handle, n, total)
    ws = torch.empty(size, dtype=torch.uint8, device="cuda")
    gT0, gY0 = torch.empty_like(T0), torch.empty_like(Y0)
    glnA = torch.empty(m.R, dtype=torch.float64, device="cuda")
    gE = torch.empty(m.R, dtype=torch.float64, device="cuda")
    st = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    rde_chem.rde_chem_advance_adjoint_ex(m.handle, dt, p, T0, Y0, n_acc, total, to_dev(gT), to_dev(gY), gT0, gY0,
                                      glnA, gE, ws, status=st)
    torch.cuda.synchronize()
    out = dict(gT0=gT0.cpu().numpy(), gY0=gY0.cpu().numpy(), glnA=glnA.cpu().numpy(), gE=gE.cpu().numpy(),
               status=st.cpu().numpy(), n_acc=n_acc.cpu().numpy(), T=T.cpu().numpy(), Y=Y.cpu().numpy())
    m.close()
    return out


def cotangents(seed, K, n):
    g = synth.normal(seed, "cot", (K + 1) * n).reshape(K + 1, n)
    return g[K].copy(), g[:K].copy()


def _oracle_cells(mech, cells, dt, opts=None):
    o = oracle.Oracle(mech.to_text())
    rec = []
    for i in range(cells.n):
        y0 = np.append(cells.Y[:, i], cells.T[i])
        rc, y1, steps = oracle.record(o, cells.p[i], y0, dt, opts)
        rec.append((rc, y0, steps))
    return o, rec


def test_adjoint_identity_and_state_gradients(h2mech):
    cells = synth.uniform_cells(h2mech, 24, seed=1001)
    gT, gY = cotangents(2001, h2mech.K, cells.n)
    g = gpu_adjoint(h2mech, cells, 1e-8, gT, gY)
    assert (g["status"] == 0).all()
    o, rec = _oracle_cells(h2mech, cells, 1e-8)
    same = [i for i in range(cells.n) if len(rec[i][2]) == g["n_acc"][i]]
    assert len(same) >= cells.n - 2
    R, N = h2mech.R, h2mech.K + 1
    dlnA = synth.uniform(5, "dlnA", R) - 0.5
    dE = (synth.uniform(5, "dE", R) - 0.5) * 1e3
    lhs = rhs = 0.0
    for i in same:
        _, y0, steps = rec[i]
        gbar = np.append(gY[:, i], gT[i])
        dy0 = (synth.uniform(6 + i, "dy0", N) - 0.5) * np.append(np.full(N - 1, 1e-3), 10.0)
        _, t = oracle.tangent(o, cells.p[i], y0, steps, dy0=dy0, dlnA=dlnA, dE=dE)
        lhs += gbar @ t
        rhs += np.append(g["gY0"][:, i], g["gT0"][i]) @ dy0
        # per-cell state gradient: column-by-column against the tangent (N directions)
        for j in range(N):
            e = np.zeros(N)
            e[j] = 1.0
            _, tj = oracle.tangent(o, cells.p[i], y0, steps, dy0=e)
            gj = g["gY0"][j, i] if j < N - 1 else g["gT0"][i]
            mag = np.abs(gbar * tj).sum()      # size of the terms (robust to cancellation)
            assert abs(gbar @ tj - gj) <= 1e-7 * mag + 1e-300, (i, j, gbar @ tj, gj)
    if len(same) == cells.n:
        rhs += g["glnA"] @ dlnA + g["gE"] @ dE
        assert abs(lhs - rhs) <= 1e-7 * max(abs(lhs), 1e-300), (lhs, rhs)


def test_parameter_gradients_vs_finite_differences(h2mech):
    cells = synth.uniform_cells(h2mech, 6, seed=1001)
    gT, gY = cotangents(2002, h2mech.K, cells.n)
    g = gpu_adjoint(h2mech, cells, 1e-8, gT, gY)
    o, rec = _oracle_cells(h2mech, cells, 1e-8)
    assert all(len(rec[i][2]) == g["n_acc"][i] for i in range(cells.n))
    R = h2mech.R
    mm = rde_chem.Mechanism(h2mech.to_text())
    _, E0 = rde_chem.rde_mech_get_arrhenius(mm.handle, R)
    mm.close()
    for name in ("lnA", "E"):
        fds, tans, gots = [], [], []
        for r in range(R):
            # h = 1e-4 relative: the frozen replay over ~700 steps carries ~1e-12 rounding noise
            # in T, which a 1e-6 step turns into ~4e-6 relative error of the difference quotient
            h = 1e-4 if name == "lnA" else 1e-4 * max(E0[r], 1e3)
            d = np.zeros(R)
            d[r] = 1.0
            fd = tan = 0.0
            for i in range(cells.n):
                _, y0, steps = rec[i]
                gbar = np.append(gY[:, i], gT[i])
                kw = {"dlnA": h * d} if name == "lnA" else {"dE": h * d}
                kwm = {"dlnA": -h * d} if name == "lnA" else {"dE": -h * d}
                _, yp = oracle.replay(o, cells.p[i], y0, steps, **kw)
                _, ym = oracle.replay(o, cells.p[i], y0, steps, **kwm)
                fd += gbar @ ((yp - ym) / (2 * h))
                _, t = oracle.tangent(o, cells.p[i], y0, steps, **({"dlnA": d} if name == "lnA" else {"dE": d}))
                tan += gbar @ t
            fds.append(fd)
            tans.append(tan)
            gots.append(g["glnA"][r] if name == "lnA" else g["gE"][r])
        fds, tans, gots = np.array(fds), np.array(tans), np.array(gots)
        scale = np.abs(tans).max()
        # exact derivative of the same frozen map (complex step): rounding-level agreement
        assert np.abs(gots - tans).max() <= 1e-7 * scale, (name, np.abs(gots - tans).max(), scale)
        # central differences: at this h the oracle's own quotients sit within 4e-8 (lnA) and
        # 6e-7 (E, O(h^2) truncation) of its exact tangent, relative to the scale
        assert np.abs(gots - fds).max() <= 2e-6 * scale, (name, np.abs(gots - fds).max(), scale)


@pytest.mark.parametrize("mix", ["uniform", "front_heavy"])
def test_parameter_gradients_per_element(h2mech, mix):
    """Every ln A_r and E_r gradient on its own: against the oracle's complex-step
    tangent of the same frozen map, |g - t| <= 1e-6 |t| + 1e-9 max|t|; against
    central differences of the frozen replay (h = 1e-4 relative), |g - fd| <= 1e-6 |g|
    + 1e-7 max|g| (the quotients' own truncation and replay-rounding floor, see the
    tolerance reading of the adjoint).  Cells: uniform states, or the front-heavy
    adjoint workload mix (fresh, post-shock front and burnt cells at dt 1e-8)."""
    if mix == "uniform":
        cells = synth.uniform_cells(h2mech, 6, seed=1001)
    else:
        field = synth.field_cells(h2mech, 400, seed=1004, fractions=(0.25, 0.50, 0.25))
        idx = np.concatenate([np.where(field.cls == c)[0][:2] for c in (0, 1, 2)])
        cells = synth.subset(field, idx)
    dt = 1e-8
    gT, gY = cotangents(2003, h2mech.K, cells.n)
    g = gpu_adjoint(h2mech, cells, dt, gT, gY)
    assert (g["status"] == 0).all()
    o, rec = _oracle_cells(h2mech, cells, dt)
    assert all(len(rec[i][2]) == g["n_acc"][i] for i in range(cells.n))
    R = h2mech.R
    mm = rde_chem.Mechanism(h2mech.to_text())
    _, E0 = rde_chem.rde_mech_get_arrhenius(mm.handle, R)
    mm.close()
    for name in ("lnA", "E"):
        tans, fds = np.zeros(R), np.zeros(R)
        for r in range(R):
            h = 1e-4 if name == "lnA" else 1e-4 * max(E0[r], 1e3)
            d = np.zeros(R)
            d[r] = 1.0
            for i in range(cells.n):
                _, y0, steps = rec[i]
                gbar = np.append(gY[:, i], gT[i])
                q = []
                for hh in (h, 0.5 * h):
                    kp = {"dlnA": hh * d} if name == "lnA" else {"dE": hh * d}
                    km = {"dlnA": -hh * d} if name == "lnA" else {"dE": -hh * d}
                    _, yp = oracle.replay(o, cells.p[i], y0, steps, **kp)
                    _, ym = oracle.replay(o, cells.p[i], y0, steps, **km)
                    q.append(gbar @ ((yp - ym) / (2 * hh)))
                fds[r] += (4.0 * q[1] - q[0]) / 3.0
                _, t = oracle.tangent(o, cells.p[i], y0, steps, **({"dlnA": d} if name == "lnA" else {"dE": d}))
                tans[r] += gbar @ t
        got = g["glnA"] if name == "lnA" else g["gE"]
        st = np.abs(tans).max()
        bad = np.abs(got - tans) > 1e-6 * np.abs(tans) + 1e-9 * st
        assert not bad.any(), (name, np.where(bad)[0], got[bad], tans[bad])
        sg = np.abs(got).max()
        bad = np.abs(got - fds) > 1e-6 * np.abs(got) + 1e-6 * sg
        assert not bad.any(), (name, np.where(bad)[0], got[bad], fds[bad])


def test_adjoint_deterministic(h2mech):
    cells = synth.field_cells(h2mech, 3000, seed=1004)
    gT, gY = cotangents(2003, h2mech.K, cells.n)
    a = gpu_adjoint(h2mech, cells, 5e-9, gT, gY)
    b = gpu_adjoint(h2mech, cells, 5e-9, gT, gY)
    assert (a["status"] == 0).all()
    assert np.isfinite(a["gT0"]).all() and np.isfinite(a["glnA"]).all() and np.isfinite(a["gE"]).all()
    for k in ("gT0", "gY0", "glnA", "gE"):
        assert np.array_equal(a[k], b[k]), k


@pytest.mark.parametrize("stages", [False, True])
@pytest.mark.parametrize("name", ["troe", "threebody_eff"])
def test_adjoint_falloff_and_efficiencies(name, stages):
    if name == "troe":
        mech = synth.isomer_mechanism(kind="TROE", reversible=True, A=3e5, b=0.3, E=40.0,
                                      low=(4e12, -0.5, 10.0), troe=(0.4, 300.0, 1800.0, 5000.0))
        mech.reactions[0].eff = {"X2": 2.0, "A": 0.7}
    else:
        mech = synth.isomer_mechanism(kind="THREEBODY", reversible=True, A=2e10, b=0.2, E=20.0)
        mech.reactions[0].eff = {"X2": 2.5}
    n = 8
    cells = synth.CellState(np.full(n, 1e5), np.linspace(1100.0, 1500.0, n),
                            np.repeat(np.array([[0.5], [0.2], [0.3]]), n, axis=1), np.zeros(n, np.int8))
    gT, gY = cotangents(2004, mech.K, n)
    dt = 2e-5
    g = gpu_adjoint(mech, cells, dt, gT, gY, rtol=1e-9, atol=1e-14, stages=stages)
    o, rec = _oracle_cells(mech, cells, dt, oracle.default_opts(rtol=1e-9, atol=1e-14))
    assert all(len(rec[i][2]) == g["n_acc"][i] for i in range(n))
    tA = tE = 0.0
    for i in range(n):
        _, y0, steps = rec[i]
        gbar = np.append(gY[:, i], gT[i])
        _, t = oracle.tangent(o, cells.p[i], y0, steps, dlnA=[1.0])
        tA += gbar @ t
        _, t = oracle.tangent(o, cells.p[i], y0, steps, dE=[1.0])
        tE += gbar @ t
        for j in range(mech.K + 1):
            e = np.zeros(mech.K + 1)
            e[j] = 1.0
            _, tj = oracle.tangent(o, cells.p[i], y0, steps, dy0=e)
            gj = g["gY0"][j, i] if j < mech.K else g["gT0"][i]
            mag = np.abs(gbar * tj).sum()
            assert abs(gbar @ tj - gj) <= 1e-7 * mag + 1e-300, (name, i, j)
    assert abs(g["glnA"][0] - tA) <= 1e-7 * abs(tA)
    assert abs(g["gE"][0] - tE) <= 1e-7 * abs(tE)


def test_autograd_function(h2mech):
    library()
    cells = synth.uniform_cells(h2mech, 64, seed=1001)
    m = rde_chem.Mechanism(h2mech.to_text())
    lnA0, E0 = rde_chem.rde_mech_get_arrhenius(m.handle, m.R)
    p, T0, Y0 = to_dev(cells.p), to_dev(cells.T).requires_grad_(True), to_dev(cells.Y).requires_grad_(True)
    lnA = torch.tensor(lnA0, device="cuda", requires_grad=True)
    E = torch.tensor(E0, device="cuda", requires_grad=True)
    T, Y, st = autograd.chem_step(m, 1e-8, p, T0, Y0, lnA, E)
    gT, gY = cotangents(2005, h2mech.K, cells.n)
    loss = (T * to_dev(gT)).sum() + (Y * to_dev(gY)).sum()
    loss.backward()
    d = gpu_adjoint(h2mech, cells, 1e-8, gT, gY)
    assert np.array_equal(T0.grad.cpu().numpy(), d["gT0"])
    assert np.array_equal(Y0.grad.cpu().numpy(), d["gY0"])
    assert np.array_equal(lnA.grad.cpu().numpy(), d["glnA"])
    assert np.array_equal(E.grad.cpu().numpy(), d["gE"])
    # a changed parameter reaches the forward step
    lnA2 = lnA.detach().clone()
    lnA2[0] += 0.5
    T2, _, _ = autograd.chem_step(m, 1e-8, p, T0.detach(), Y0.detach(), lnA2, E.detach())
    assert not torch.equal(T2, T.detach())
    m.close()


def _adjoint_at(text, lnA, E, dt, p, T0, Y0, gT, gY):
    """Forward and adjoint of one step through the C ABI at explicit Arrhenius parameters."""
    m = rde_chem.Mechanism(text)
    rde_chem.rde_mech_set_arrhenius(m.handle, lnA, E)
    n = int(T0.shape[0])
    T, Y = T0.clone(), Y0.clone()
    n_acc = torch.zeros(n, dtype=torch.int32, device="cuda")
    rde_chem.rde_chem_advance_ex(m.handle, dt, cells=rde_chem.make_block(p, T, Y, n_acc=n_acc), threads_per_cta=128)
    total = int(n_acc.sum().item())
    ws = torch.empty(rde_chem.rde_chem_adjoint_workspace_steps(m.handle, n, total), dtype=torch.uint8, device="cuda")
    gT0, gY0 = torch.empty_like(T0), torch.empty_like(Y0)
    glnA = torch.empty(m.R, dtype=torch.float64, device="cuda")
    gE = torch.empty(m.R, dtype=torch.float64, device="cuda")
    rde_chem.rde_chem_advance_adjoint_ex(m.handle, dt, p, T0, Y0, n_acc, total, gT, gY, gT0, gY0, glnA, gE, ws)
    torch.cuda.synchronize()
    m.close()
    return T, Y, gT0, gY0, glnA, gE


def test_autograd_two_steps_with_different_parameters(h2mech):
    """Two chained steps on one Mechanism with different ln A / E: each backward runs at
    the parameters its own forward used (not the ones the tables hold at backward time),
    and the tables afterwards hold what they held before backward."""
    library()
    cells = synth.uniform_cells(h2mech, 32, seed=1001)
    text = h2mech.to_text()
    m = rde_chem.Mechanism(text)
    lnA0, E0 = rde_chem.rde_mech_get_arrhenius(m.handle, m.R)
    lnA_b = lnA0 + 0.3 * (synth.uniform(7, "dlnA", m.R) - 0.5)
    E_b = E0 * (1.0 + 0.02 * (synth.uniform(7, "dE", m.R) - 0.5))
    p, T0, Y0 = to_dev(cells.p), to_dev(cells.T).requires_grad_(True), to_dev(cells.Y).requires_grad_(True)
    a_lnA = torch.tensor(lnA0, device="cuda", requires_grad=True)
    a_E = torch.tensor(E0, device="cuda", requires_grad=True)
    b_lnA = torch.tensor(lnA_b, device="cuda", requires_grad=True)
    b_E = torch.tensor(E_b, device="cuda", requires_grad=True)
    dt = 1e-8
    T1, Y1, _ = autograd.chem_step(m, dt, p, T0, Y0, a_lnA, a_E)
    T2, Y2, _ = autograd.chem_step(m, dt, p, T1, Y1, b_lnA, b_E)
    gT, gY = cotangents(2007, h2mech.K, cells.n)
    gT, gY = to_dev(gT), to_dev(gY)
    ((T2 * gT).sum() + (Y2 * gY).sum()).backward()
    after = rde_chem.rde_mech_get_arrhenius(m.handle, m.R)
    assert np.array_equal(after[0], lnA_b) and np.array_equal(after[1], E_b)
    m.close()
    # reference: the two adjoints through the C ABI, each at its own parameters
    T1r, Y1r, _, _, _, _ = _adjoint_at(text, lnA0, E0, dt, p, T0.detach(), Y0.detach(), gT, gY)
    assert torch.equal(T1r, T1.detach()) and torch.equal(Y1r, Y1.detach())
    _, _, gT1, gY1, glnA_b, gE_b = _adjoint_at(text, lnA_b, E_b, dt, p, T1r, Y1r, gT, gY)
    _, _, gT0r, gY0r, glnA_a, gE_a = _adjoint_at(text, lnA0, E0, dt, p, T0.detach(), Y0.detach(), gT1, gY1)
    assert torch.equal(b_lnA.grad, glnA_b) and torch.equal(b_E.grad, gE_b)
    assert torch.equal(a_lnA.grad, glnA_a) and torch.equal(a_E.grad, gE_a)
    assert torch.equal(T0.grad, gT0r) and torch.equal(Y0.grad, gY0r)
    # the first step's gradient at the second step's parameters would differ
    _, _, _, _, glnA_wrong, _ = _adjoint_at(text, lnA_b, E_b, dt, p, T0.detach(), Y0.detach(), gT1, gY1)
    assert not torch.equal(glnA_wrong, glnA_a)


@pytest.mark.parametrize("K", [9, 3])
def test_stage_checkpoints_match_recompute(h2mech, K):
    """Stage checkpoints (the re-integration stores each accepted step's LU factors and
    stages) and stage recompute differentiate the same discrete map: the gradients agree
    to rounding (the recomputed stages are not bitwise the stored ones), and with
    checkpoints the result is deterministic."""
    if K == 9:
        mech, cells, dt = h2mech, synth.field_cells(h2mech, 3000, seed=1004, fractions=(0.25, 0.5, 0.25)), 1e-8
    else:
        mech, cells, dt = small_case("troe", n=200)
    gT, gY = cotangents(2007, mech.K, cells.n)
    a = gpu_adjoint(mech, cells, dt, gT, gY)
    b = gpu_adjoint(mech, cells, dt, gT, gY, stages=True)
    c = gpu_adjoint(mech, cells, dt, gT, gY, stages=True)
    assert (a["status"] == 0).all() and (b["status"] == 0).all()
    for k in ("gT0", "gY0", "glnA", "gE"):
        assert np.array_equal(b[k], c[k]), k
        scale = np.abs(a[k]).max()
        assert np.abs(a[k] - b[k]).max() <= 1e-9 * scale, (k, np.abs(a[k] - b[k]).max() / scale)


def test_undersized_total_steps_is_reported_not_overrun(h2mech):
    """A total_steps below the sum of n_steps sizes a smaller pool: the cells whose records
    would end beyond it report RDE_CELL_ADJ_MISMATCH with zero gradients, the others are
    differentiated as usual, and nothing is written outside the workspace."""
    cells = synth.uniform_cells(h2mech, 64, seed=1008)
    gT, gY = cotangents(2008, h2mech.K, cells.n)
    full = gpu_adjoint(h2mech, cells, 1e-8, gT, gY, stages=True)
    total = int(full["n_acc"].sum())
    part = gpu_adjoint(h2mech, cells, 1e-8, gT, gY, stages=True, total_steps=total // 2)
    ends = np.cumsum(full["n_acc"])
    fits = ends <= total // 2
    assert fits.any() and (~fits).any()
    assert (part["status"][~fits] == 5).all() and (part["status"][fits] == 0).all()
    assert (part["gT0"][~fits] == 0).all() and (part["gY0"][:, ~fits] == 0).all()
    assert np.array_equal(part["gT0"][fits], full["gT0"][fits])
    assert np.array_equal(part["gY0"][:, fits], full["gY0"][:, fits])


def test_checkpointed_workspace_size(h2mech):
    library()
    m = rde_chem.Mechanism(h2mech.to_text())
    N = h2mech.K + 1
    for n, total in ((1, 1), (1000, 123457), (262144, 153469015)):
        a = rde_chem.rde_chem_adjoint_workspace_steps(m.handle, n, total)
        b = rde_chem.rde_chem_adjoint_workspace_checkpointed(m.handle, n, total)
        extra = total * (N * N + 4 * N + 1) * 8
        assert extra <= b - a < extra + 256
    assert rde_chem.rde_chem_adjoint_workspace_checkpointed(m.handle, -1, 5) == 0
    m.close()


@pytest.mark.parametrize("nd", ["1", "2"])
def test_multi_direction_second_derivatives(h2mech, monkeypatch, nd):
    """The specialised reverse kernel evaluates the four stages' second-derivative terms
    in one pass that carries four directions (the default) or, by RDE_JIT_HVP_DIRECTIONS,
    one pass per stage (plain dual numbers) or two passes of two.  All give the same
    gradients up to rounding order."""
    cells = synth.field_cells(h2mech, 2000, seed=1009, fractions=(0.25, 0.5, 0.25))
    gT, gY = cotangents(2009, h2mech.K, cells.n)
    monkeypatch.delenv("RDE_JIT_HVP_DIRECTIONS", raising=False)
    a = gpu_adjoint(h2mech, cells, 1e-8, gT, gY, stages=True)
    monkeypatch.setenv("RDE_JIT_HVP_DIRECTIONS", nd)
    b = gpu_adjoint(h2mech, cells, 1e-8, gT, gY, stages=True)
    assert (a["status"] == 0).all() and (b["status"] == 0).all()
    for k in ("gT0", "gY0", "glnA", "gE"):
        scale = np.abs(a[k]).max()
        assert np.abs(a[k] - b[k]).max() <= 1e-11 * scale, (k, np.abs(a[k] - b[k]).max() / scale)
