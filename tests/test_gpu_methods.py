"""GPU parity of the second integrator (ROS2, two-stage L-stable Rosenbrock of order 2(1))
against the oracle's ROS2, and the method switch of the C ABI.

Both sides integrate with the same transformed coefficients, the same RMS norm and the
same controller (exponent 1/2 for the order-1 embedded estimate), so they differ only by
rounding, as for RODAS3; at rtol 1e-8 the parity bounds are the same.
"""
import numpy as np
import pytest
import torch

import oracle
from gpu_util import assert_parity, library, run_gpu, run_oracle, to_dev
from paper_2508_16105_gb300 import rde_chem, synth

pytestmark = pytest.mark.gpu

ROS2, RODAS3 = rde_chem.RDE_METHOD_ROS2, rde_chem.RDE_METHOD_RODAS3
PLAIN, QUEUE, BLOCK = rde_chem.RDE_SCHED_PLAIN, rde_chem.RDE_SCHED_QUEUE, rde_chem.RDE_SCHED_BLOCK
ERR_ARG, ERR_UNSUPPORTED = -2, -6


@pytest.fixture(scope="module")
def mech():
    library()
    return synth.h2_air_mechanism(16105)


def test_ros2_uniform_cells(mech):
    """1024 uniform cells at the parity tolerances (rtol 1e-8): about 10^4 ROS2 steps a cell."""
    cells = synth.uniform_cells(mech, 1024, seed=1001)
    g = run_gpu(mech, cells, 1e-8, method=ROS2)
    o = run_oracle(mech, cells, 1e-8, method=oracle.METHOD_ROS2)
    assert_parity(g, o)
    assert (g["status"] == 0).all()
    assert abs(g["n_acc"].sum() / o["n_acc"].sum() - 1) < 1e-3


@pytest.mark.parametrize("rtol", [1e-6, 1e-4])
def test_ros2_field_cells(mech, rtol):
    """Fresh, front and burnt cells at looser tolerances, against the oracle at the same rtol."""
    cells = synth.field_cells(mech, 2000, seed=1002, fractions=(0.3, 0.4, 0.3))
    g = run_gpu(mech, cells, 5e-9, rtol=rtol, method=ROS2)
    o = run_oracle(mech, cells, 5e-9, rtol=rtol, method=oracle.METHOD_ROS2)
    # a step decision flipped by rounding moves a cell by up to about rtol
    assert_parity(g, o, T_tol=max(1e-6, 10 * rtol), Y_tol=max(1e-9, 10 * rtol))
    assert abs(g["n_acc"].sum() / o["n_acc"].sum() - 1) < 1e-3


def test_ros2_schedules_and_kernels(mech):
    """PLAIN and QUEUE schedules give bitwise the same results with each kernel; the specialised
    and precompiled kernels (constants folded differently) agree to rounding."""
    cells = synth.field_cells(mech, 777, seed=1003, fractions=(0.3, 0.4, 0.3))
    runs = {(s, f): run_gpu(mech, cells, 5e-9, rtol=1e-6, method=ROS2, schedule=s, flags=f)
            for s in (PLAIN, QUEUE) for f in (0, rde_chem.RDE_LOAD_GENERIC)}
    for f in (0, rde_chem.RDE_LOAD_GENERIC):
        for k in ("T", "Y", "status", "n_acc", "n_rej"):
            assert np.array_equal(runs[(PLAIN, f)][k], runs[(QUEUE, f)][k]), (f, k)
    assert_parity(runs[(QUEUE, 0)], runs[(QUEUE, rde_chem.RDE_LOAD_GENERIC)], T_tol=1e-5, Y_tol=1e-5)


def test_ros2_and_rodas3_agree_within_tolerance(mech):
    """The two methods reach the same state to within their tolerance; ROS2 needs more steps."""
    cells = synth.uniform_cells(mech, 512, seed=1004)
    a = run_gpu(mech, cells, 1e-8, method=RODAS3)
    b = run_gpu(mech, cells, 1e-8, method=ROS2)
    assert not np.array_equal(a["T"], b["T"])
    assert np.max(np.abs(a["T"] - b["T"]) / a["T"]) < 1e-8
    assert np.max(np.abs(a["Y"] - b["Y"])) < 1e-8
    assert b["n_acc"].sum() > 5 * a["n_acc"].sum()


def test_ros2_conserves_mass_and_elements(mech):
    cells = synth.field_cells(mech, 4096, seed=1005)
    Y0 = cells.Y.copy()
    g = run_gpu(mech, cells, 5e-9, rtol=1e-6, method=ROS2)
    assert (g["status"] == 0).all()
    assert np.max(np.abs(g["Y"].sum(axis=0) - Y0.sum(axis=0))) < 5e-12
    E = np.array([[s.comp.get(e, 0) / s.W for s in mech.species] for e in mech.elements])
    assert np.max(np.abs(E @ g["Y"] - E @ Y0)) < 5e-12


def test_method_switch_on_one_handle(mech):
    """set_options switches the method of a loaded handle; switching back gives RODAS3 bitwise."""
    library()
    cells = synth.uniform_cells(mech, 300, seed=1006)
    m = rde_chem.Mechanism(mech.to_text())
    outs = []
    for meth in (RODAS3, ROS2, RODAS3):
        o = rde_chem.rde_chem_default_options()
        o.method = meth
        rde_chem.rde_chem_set_options(m.handle, o)
        p, T, Y = to_dev(cells.p), to_dev(cells.T), to_dev(cells.Y)
        rde_chem.rde_chem_advance(m.handle, cells.n, p, T, Y, 1e-8)
        torch.cuda.synchronize()
        outs.append(T.cpu().numpy())
    assert np.array_equal(outs[0], outs[2]) and not np.array_equal(outs[0], outs[1])
    m.close()


def test_ros2_unsupported_paths(mech):
    """The CTA-per-cell kernel and the adjoint integrate RODAS3 only: ROS2 there is refused on
    the host before any launch; an unknown method is an argument error."""
    library()
    m = rde_chem.Mechanism(mech.to_text(), method=ROS2)
    cells = synth.uniform_cells(mech, 8, seed=1007)
    p, T, Y = to_dev(cells.p), to_dev(cells.T), to_dev(cells.Y)
    blk = rde_chem.make_block(p, T, Y, n=cells.n, ldY=cells.n)
    with pytest.raises(rde_chem.RdeError) as e:
        rde_chem.rde_chem_advance_ex(m.handle, 1e-8, cells=blk, schedule=BLOCK)
    assert e.value.code == ERR_UNSUPPORTED
    n = cells.n
    n_acc = torch.ones(n, dtype=torch.int32, device="cuda")
    ws = torch.empty(rde_chem.rde_chem_adjoint_workspace_steps(m.handle, n, n), dtype=torch.uint8, device="cuda")
    gT0, gY0 = torch.empty_like(T), torch.empty_like(Y)
    g_lnA, g_E = (torch.empty(m.R, dtype=torch.float64, device="cuda") for _ in range(2))
    with pytest.raises(rde_chem.RdeError) as e:
        rde_chem.rde_chem_advance_adjoint_ex(m.handle, 1e-8, p, T, Y, n_acc, n, torch.ones_like(T),
                                          torch.zeros_like(Y), gT0, gY0, g_lnA, g_E, ws)
    assert e.value.code == ERR_UNSUPPORTED
    o = rde_chem.rde_chem_default_options()
    o.method = 7
    with pytest.raises(rde_chem.RdeError) as e:
        rde_chem.rde_chem_set_options(m.handle, o)
    assert e.value.code == ERR_ARG
    m.close()


def test_ros2_refused_without_a_thread_per_cell_kernel():
    """53 species: only the CTA-per-cell kernel serves the mechanism, so selecting ROS2 fails
    and leaves the handle's options unchanged."""
    library()
    big = synth.large_mechanism(16105)
    m = rde_chem.Mechanism(big.to_text())
    o = rde_chem.rde_chem_default_options()
    o.method = ROS2
    with pytest.raises(rde_chem.RdeError) as e:
        rde_chem.rde_chem_set_options(m.handle, o)
    assert e.value.code == ERR_UNSUPPORTED
    assert rde_chem.rde_chem_get_options(m.handle).method == RODAS3
    m.close()


EXTRAP = rde_chem.RDE_METHOD_EXTRAP


def test_extrapolation_uniform_cells(mech):
    """The third method (linearly implicit Euler extrapolated to order 3) against the
    oracle's same method at the parity tolerances (rtol 1e-8), specialised kernel."""
    cells = synth.uniform_cells(mech, 512, seed=1001)
    g = run_gpu(mech, cells, 1e-8, method=EXTRAP)
    o = run_oracle(mech, cells, 1e-8, method=oracle.METHOD_EXTRAP)
    assert_parity(g, o)
    assert (g["status"] == 0).all()
    assert abs(g["n_acc"].sum() / o["n_acc"].sum() - 1) < 1e-3


@pytest.mark.parametrize("flags", [0, rde_chem.RDE_LOAD_GENERIC])
def test_extrapolation_field_cells(mech, flags):
    """Fresh, front and burnt cells at rtol 1e-6 with the specialised and the precompiled
    kernels, against the oracle at the same rtol; mass conserved."""
    cells = synth.field_cells(mech, 1500, seed=1002, fractions=(0.3, 0.4, 0.3))
    g = run_gpu(mech, cells, 5e-9, rtol=1e-6, method=EXTRAP, flags=flags)
    o = run_oracle(mech, cells, 5e-9, rtol=1e-6, method=oracle.METHOD_EXTRAP)
    assert_parity(g, o, T_tol=1e-5, Y_tol=1e-5)
    assert abs(g["n_acc"].sum() / o["n_acc"].sum() - 1) < 2e-3
    assert np.max(np.abs(g["Y"].sum(axis=0) - cells.Y.sum(axis=0))) < 5e-12


def test_extrapolation_queue_only_and_agrees_with_rodas3(mech):
    """The plain schedule is refused for the extrapolation method (its Jacobian scratch is
    per resident lane); its result agrees with RODAS3 within the tolerance."""
    library()
    m = rde_chem.Mechanism(mech.to_text(), method=EXTRAP)
    cells = synth.uniform_cells(mech, 64, seed=1008)
    p, T, Y = to_dev(cells.p), to_dev(cells.T), to_dev(cells.Y)
    blk = rde_chem.make_block(p, T, Y, n=cells.n, ldY=cells.n)
    with pytest.raises(rde_chem.RdeError) as e:
        rde_chem.rde_chem_advance_ex(m.handle, 1e-8, cells=blk, schedule=PLAIN)
    assert e.value.code == ERR_UNSUPPORTED
    m.close()
    a = run_gpu(mech, cells, 1e-8, method=RODAS3)
    b = run_gpu(mech, cells, 1e-8, method=EXTRAP)
    assert np.max(np.abs(a["T"] - b["T"]) / a["T"]) < 1e-7
    assert np.max(np.abs(a["Y"] - b["Y"])) < 1e-8
