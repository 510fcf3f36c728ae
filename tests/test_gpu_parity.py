"""GPU parity: the sm_103a chemistry step against the CPU oracle, cell by cell.

Tolerances (at rtol 1e-8, atol 1e-12): |dT|/T <= 1e-6 and |dY_k| <= 1e-9; the
per-cell status must match exactly.  Both sides run the same algorithm with the
same controller, so they differ only by rounding (and the rare step decision
that rounding flips); the oracle's own global error against a tight Radau run
is about 100x smaller than these bounds (tests/test_oracle_accuracy.py).
"""
import numpy as np
import pytest
import torch

from gpu_util import SMALL_CASES, assert_parity, library, run_gpu, run_oracle, small_case, to_dev
from paper_2508_16105_gb300 import rde_chem, synth

pytestmark = pytest.mark.gpu

PLAIN, QUEUE = rde_chem.RDE_SCHED_PLAIN, rde_chem.RDE_SCHED_QUEUE


@pytest.fixture(scope="module")
def mech():
    library()
    return synth.h2_air_mechanism(16105)


@pytest.fixture(scope="module")
def c1_cells(mech):
    return synth.uniform_cells(mech, 4096, seed=1001)


@pytest.fixture(scope="module")
def c1_oracle(mech, c1_cells):
    return run_oracle(mech, c1_cells, 1e-8)


def test_uniform_4096_cells(mech, c1_cells, c1_oracle):
    g = run_gpu(mech, c1_cells, 1e-8)
    dT, dY = assert_parity(g, c1_oracle)
    assert (g["status"] == 0).all()
    assert g["stats"]["cells"] == 4096
    assert g["stats"]["accepted"] == int(g["n_acc"].sum())
    assert g["stats"]["rejected"] == int(g["n_rej"].sum())
    # step counts agree closely with the oracle's (same controller, rounding-level differences)
    assert abs(g["stats"]["accepted"] / c1_oracle["n_acc"].sum() - 1) < 1e-3


def test_plain_equals_queue_bitwise(mech, c1_cells, c1_oracle):
    """The 128-thread kernels give the same bits on either schedule and launch shape; the
    wide 256-thread queue kernel (the AUTO choice here) matches the oracle and agrees
    with them to rounding."""
    a = run_gpu(mech, c1_cells, 1e-8, schedule=PLAIN)
    b = run_gpu(mech, c1_cells, 1e-8, schedule=QUEUE, threads=128)
    c = run_gpu(mech, c1_cells, 1e-8, schedule=QUEUE, ctas_per_sm=1, threads=128)
    for k in ("T", "Y", "status", "n_acc", "n_rej"):
        assert np.array_equal(a[k], b[k]), k
        assert np.array_equal(a[k], c[k]), k
    w = run_gpu(mech, c1_cells, 1e-8, schedule=QUEUE, threads=256)
    assert_parity(w, c1_oracle)
    assert np.array_equal(w["status"], a["status"])
    assert np.abs(w["T"] / a["T"] - 1).max() <= 1e-9
    assert np.abs(w["Y"] - a["Y"]).max() <= 1e-11


def test_deterministic(mech, c1_cells):
    idx = np.arange(512)
    cells = synth.subset(c1_cells, idx)
    a = run_gpu(mech, cells, 1e-8)
    b = run_gpu(mech, cells, 1e-8)
    assert np.array_equal(a["T"], b["T"]) and np.array_equal(a["Y"], b["Y"])


@pytest.mark.parametrize("n", [1, 31, 33, 129, 1000])
def test_ragged_sizes(mech, c1_cells, c1_oracle, n):
    idx = np.arange(n) * 3 % 4096
    cells = synth.subset(c1_cells, idx)
    for sched in (PLAIN, QUEUE):
        g = run_gpu(mech, cells, 1e-8, schedule=sched)
        o = {k: (v[..., idx] if v is not None else None) for k, v in c1_oracle.items()}
        assert_parity(g, o)


def test_empty_call(mech):
    library()
    m = rde_chem.Mechanism(mech.to_text())
    rde_chem.rde_chem_advance(m.handle, 0, None, None, None, 1e-8)
    assert rde_chem.rde_chem_get_stats(m.handle)["cells"] == 0
    with pytest.raises(rde_chem.RdeError):
        rde_chem.rde_chem_advance(m.handle, -1, None, None, None, 1e-8)
    T = torch.ones(4, dtype=torch.float64, device="cuda")
    with pytest.raises(rde_chem.RdeError):
        rde_chem.rde_chem_advance(m.handle, 4, T, T, T, 0.0)
    m.close()


def test_bad_states_untouched(mech, c1_cells):
    cells = synth.subset(c1_cells, np.arange(64))
    cells.T[3] = np.nan
    cells.T[7] = -5.0
    cells.p[11] = 0.0
    cells.Y[2, 13] = np.inf
    g = run_gpu(mech, cells, 1e-8)
    bad = [3, 7, 11, 13]
    assert (g["status"][bad] == 3).all()
    good = np.setdiff1d(np.arange(64), bad)
    assert (g["status"][good] == 0).all()
    assert np.array_equal(g["T"][[7]], [-5.0]) and np.isnan(g["T"][3])
    assert np.array_equal(g["Y"][:, 13], cells.Y[:, 13])
    o = run_oracle(mech, cells, 1e-8)
    assert_parity(g, o)


def test_max_substeps_keeps_last_accepted(mech, c1_cells):
    cells = synth.subset(c1_cells, np.arange(200))
    g = run_gpu(mech, cells, 1e-8, max_substeps=40)
    o = run_oracle(mech, cells, 1e-8, max_substeps=40)
    assert (g["status"] == 1).sum() > 100
    assert_parity(g, o)
    assert np.array_equal(g["n_acc"] + g["n_rej"], o["n_acc"] + o["n_rej"])


def test_h_hint_round_trip(mech, c1_cells):
    cells = synth.subset(c1_cells, np.arange(256))
    hint0 = np.full(256, 3e-13)
    hint0[::7] = 0.0          # zero hint: start from dt
    g = run_gpu(mech, cells, 1e-8, hint=hint0)
    o = run_oracle(mech, cells, 1e-8, hint=hint0)
    assert_parity(g, o)
    # the proposed next step scales with err^(-1/3) of a small, cancellation-prone error
    # estimate, so it carries more relative rounding noise than the state itself
    assert np.abs(g["hint"] / o["hint"] - 1).max() < 1e-3


@pytest.mark.parametrize("threads", [0, 256])
def test_strided_Y_and_block_table(mech, c1_cells, threads):
    """Padded blocks (one empty) in a block table with a reversed queue order, on the
    128-thread kernels (0) and on the wide queue kernel (256)."""
    library()
    sizes = [300, 0, 77, 1200, 5]
    n = sum(sizes)
    cells = synth.subset(c1_cells, np.arange(n))
    ref = run_oracle(mech, cells, 1e-8)
    m = rde_chem.Mechanism(mech.to_text())
    blocks, keep, off = [], [], 0
    for s in sizes:
        ld = s + 3    # padded leading dimension
        Yp = torch.zeros((m.K, max(ld, 1)), dtype=torch.float64, device="cuda")
        Yp[:, :s] = to_dev(cells.Y[:, off:off + s])
        p, T = to_dev(cells.p[off:off + s]), to_dev(cells.T[off:off + s])
        st = torch.full((max(s, 1),), -1, dtype=torch.int32, device="cuda")
        keep.append((p, T, Yp, st, off, s))
        blocks.append(rde_chem.make_block(p, T, Yp, status=st, n=s, ldY=ld))
        off += s
    table = torch.frombuffer(bytearray(rde_chem.block_table_bytes(blocks)), dtype=torch.uint8).cuda()
    order = torch.arange(n - 1, -1, -1, dtype=torch.int64, device="cuda")   # reversed queue order
    rde_chem.rde_chem_advance_ex(m.handle, 1e-8, blocks=table, n_blocks=len(sizes), n_total=n, order=order,
                                 threads_per_cta=threads)
    assert rde_chem.rde_chem_get_stats(m.handle)["cells"] == n
    for p, T, Yp, st, o0, s in keep:
        if s == 0:
            continue
        g = dict(T=T.cpu().numpy(), Y=Yp[:, :s].cpu().numpy(), status=st[:s].cpu().numpy())
        r = dict(T=ref["T"][o0:o0 + s], Y=ref["Y"][:, o0:o0 + s], status=ref["status"][o0:o0 + s])
        assert_parity(g, r)
        assert (Yp[:, s:] == 0).all()   # padding untouched
    m.close()


@pytest.mark.parametrize("name", SMALL_CASES)
def test_small_mechanisms(name):
    library()
    mech, cells, dt = small_case(name)
    g = run_gpu(mech, cells, dt, rtol=1e-9, atol=1e-15)
    o = run_oracle(mech, cells, dt, rtol=1e-9, atol=1e-15)
    assert (g["status"] == 0).all()
    assert_parity(g, o, T_tol=1e-9, Y_tol=1e-10)


def test_field_full_size_sampled(mech):
    """The 2,097,152-cell RDE-like field in the benchmark's launch (queue schedule), sampled."""
    cells = synth.field_cells(mech, 2097152, seed=1002)
    g = run_gpu(mech, cells, 5e-9)
    assert (g["status"] == 0).all()
    rng_idx = synth.sample_indices(77, cells.n, 192)
    costly = np.argsort(g["n_acc"] + g["n_rej"])[-64:]
    idx = np.unique(np.concatenate([rng_idx, costly]))
    sub = synth.subset(cells, idx)
    o = run_oracle(mech, sub, 5e-9)
    gs = dict(T=g["T"][idx], Y=g["Y"][:, idx], status=g["status"][idx])
    assert_parity(gs, o)
    # the sampled cells cover all three classes
    assert set(np.unique(cells.cls[idx]).tolist()) == {0, 1, 2}
    # every cell: the step conserves mass and each element exactly in exact arithmetic
    # (element-balanced reactions; E^T W^-1 J_Y = 0 makes each Rosenbrock stage conserve
    # them too), so only rounding over ~280 substeps remains
    assert np.abs(g["Y"].sum(axis=0) - cells.Y.sum(axis=0)).max() <= 5e-12
    elems = mech.elements
    Z = np.array([[s_.comp.get(e, 0) * synth.ATOMIC_MASS[e] / s_.W for s_ in mech.species] for e in elems])
    assert np.abs(Z @ g["Y"] - Z @ cells.Y).max() <= 5e-12
