"""GPU parity of the CTA-per-cell kernel (RDE_SCHED_BLOCK; the AUTO choice for
species counts without a thread-per-cell kernel) against the CPU oracle.

The kernel sums over reactions and species in another fixed order than the
thread-per-cell kernels, so it agrees with the oracle to rounding: the same
bounds as the other parity tests apply (|dT|/T <= 1e-6, |dY_k| <= 1e-9 at rtol
1e-8, atol 1e-12; tighter for the small mechanisms) and statuses match exactly.
The 53-species, 325-reaction stress mechanism (20 three-body, 10 Troe) is the
case this kernel exists for: a 54 x 54 Jacobian and LU per cell.
"""
import numpy as np
import pytest
import torch

from gpu_util import SMALL_CASES, assert_parity, library, run_gpu, run_oracle, small_case, to_dev
from paper_2508_16105_gb300 import rde_chem, synth

pytestmark = pytest.mark.gpu

BLOCK, PLAIN, QUEUE, AUTO = rde_chem.RDE_SCHED_BLOCK, rde_chem.RDE_SCHED_PLAIN, rde_chem.RDE_SCHED_QUEUE, \
    rde_chem.RDE_SCHED_AUTO


@pytest.fixture(scope="module")
def big():
    library()
    return synth.large_mechanism()


@pytest.fixture(scope="module")
def big_cells(big):
    return synth.field_cells(big, 192, seed=1005)


@pytest.fixture(scope="module")
def big_oracle(big, big_cells):
    return run_oracle(big, big_cells, 5e-9)


def test_h2_block_kernel_vs_oracle(h2mech):
    cells = synth.uniform_cells(h2mech, 1024, seed=1001)
    g = run_gpu(h2mech, cells, 1e-8, schedule=BLOCK)
    o = run_oracle(h2mech, cells, 1e-8)
    assert (g["status"] == 0).all()
    assert_parity(g, o)
    assert g["stats"]["cells"] == 1024
    assert g["stats"]["accepted"] == int(g["n_acc"].sum())


def test_h2_block_kernel_field_front_cells(h2mech):
    cells = synth.field_cells(h2mech, 3000, seed=1002, fractions=(0.2, 0.6, 0.2))
    g = run_gpu(h2mech, cells, 5e-9, schedule=BLOCK)
    o = run_oracle(h2mech, cells, 5e-9)
    assert_parity(g, o)


@pytest.mark.parametrize("name", SMALL_CASES)
def test_small_mechanisms_block_kernel(name):
    library()
    mech, cells, dt = small_case(name)
    g = run_gpu(mech, cells, dt, rtol=1e-9, atol=1e-15, schedule=BLOCK)
    o = run_oracle(mech, cells, dt, rtol=1e-9, atol=1e-15)
    assert (g["status"] == 0).all()
    assert_parity(g, o, T_tol=1e-9, Y_tol=1e-10)


def test_large_mechanism_vs_oracle(big, big_cells, big_oracle):
    g = run_gpu(big, big_cells, 5e-9, schedule=AUTO)
    assert (g["status"] == 0).all()
    dT, dY = assert_parity(g, big_oracle)
    # same controller: accepted-step totals agree to rounding-level step decisions
    assert abs(g["n_acc"].sum() / big_oracle["n_acc"].sum() - 1) < 1e-3
    assert set(np.unique(big_cells.cls).tolist()) == {0, 1, 2}


@pytest.mark.parametrize("n", [1, 7, 33, 150])
def test_large_ragged_and_plain_queue_bitwise(big, big_cells, big_oracle, n):
    idx = np.arange(n) * 5 % big_cells.n
    cells = synth.subset(big_cells, idx)
    a = run_gpu(big, cells, 5e-9, schedule=PLAIN)
    b = run_gpu(big, cells, 5e-9, schedule=QUEUE)
    c = run_gpu(big, cells, 5e-9, schedule=QUEUE, ctas_per_sm=1)
    for k in ("T", "Y", "status", "n_acc", "n_rej"):
        assert np.array_equal(a[k], b[k]), k
        assert np.array_equal(a[k], c[k]), k
    o = {k: (v[..., idx] if v is not None else None) for k, v in big_oracle.items()}
    assert_parity(b, o)


def test_large_block_table_order_and_hint(big, big_cells):
    """Four blocks (one empty) with padded leading dimensions, a permutation and step-size hints."""
    library()
    m = rde_chem.Mechanism(big.to_text())
    sizes = [50, 0, 1, 41]
    ref = run_gpu(big, synth.subset(big_cells, np.arange(sum(sizes))), 5e-9)
    keep, blocks, o0 = [], [], 0
    for s in sizes:
        ld = s + 3
        Yp = torch.zeros(big.K, ld, dtype=torch.float64, device="cuda")
        Yp[:, :s] = to_dev(big_cells.Y[:, o0:o0 + s])
        p, T = to_dev(big_cells.p[o0:o0 + s]), to_dev(big_cells.T[o0:o0 + s])
        st = torch.full((max(s, 1),), -1, dtype=torch.int32, device="cuda")
        hint = torch.zeros(max(s, 1), dtype=torch.float64, device="cuda")
        keep.append((p, T, Yp, st, hint, s, o0))
        blocks.append(rde_chem.make_block(p, T, Yp, h_hint=hint, status=st, n=s, ldY=ld))
        o0 += s
    table = torch.frombuffer(bytearray(rde_chem.block_table_bytes(blocks)), dtype=torch.uint8).cuda()
    order = to_dev(np.argsort(synth.uniform(9, "perm", o0), kind="stable"), dtype=torch.int64)
    rde_chem.rde_chem_advance_ex(m.handle, 5e-9, blocks=table, n_blocks=len(blocks), n_total=o0,
                                 order=order, schedule=BLOCK)
    assert rde_chem.rde_chem_get_stats(m.handle)["cells"] == o0
    torch.cuda.synchronize()
    for p, T, Yp, st, hint, s, a0 in keep:
        if s == 0:
            continue
        assert np.array_equal(T.cpu().numpy(), ref["T"][a0:a0 + s])
        assert np.array_equal(Yp[:, :s].cpu().numpy(), ref["Y"][:, a0:a0 + s])
        assert (st[:s].cpu().numpy() == 0).all()
        assert (hint[:s].cpu().numpy() > 0).all()
        assert (Yp[:, s:] == 0).all()
    m.close()


def test_large_bad_state_untouched(big, big_cells):
    cells = synth.subset(big_cells, np.arange(8))
    cells.T[2] = np.nan
    cells.p[5] = -1.0
    g = run_gpu(big, cells, 5e-9)
    assert g["status"][2] == 3 and g["status"][5] == 3
    assert np.isnan(g["T"][2]) and np.array_equal(g["Y"][:, 5], cells.Y[:, 5])
    assert (np.delete(g["status"], [2, 5]) == 0).all()


def test_large_kernel_info_and_adjoint_workspace(big):
    """53 species: the CTA-per-cell adjoint serves the mechanism; its workspace holds no
    thread-per-cell lane scratch, and a too-small workspace is refused before any launch."""
    library()
    m = rde_chem.Mechanism(big.to_text())
    info = rde_chem.rde_chem_kernel_info(m.handle)
    assert info["threads_per_cta"] == 128
    assert info["max_ctas_per_sm"] >= 1
    assert 0 < info["shared_bytes"] <= 227 * 1024
    n, total = 4, 0
    need = rde_chem.rde_chem_adjoint_workspace_steps(m.handle, n, total)
    assert need < 1 << 20
    z = torch.zeros(n, dtype=torch.float64, device="cuda")
    zy = torch.zeros(big.K, n, dtype=torch.float64, device="cuda")
    na = torch.zeros(n, dtype=torch.int32, device="cuda")
    gr = torch.zeros(big.R, dtype=torch.float64, device="cuda")
    ws = torch.empty(need - 256, dtype=torch.uint8, device="cuda")
    with pytest.raises(rde_chem.RdeError) as e:
        rde_chem.rde_chem_advance_adjoint_ex(m.handle, 5e-9, z, z, zy, na, total, z, zy, z.clone(), zy.clone(), gr,
                                          gr.clone(), ws)
    assert e.value.code == -8      # RDE_ERR_WORKSPACE
    m.close()


def test_large_bench_workload_sampled(big):
    """The stress benchmark's launch: 16,384 field cells (a 1/64 sample of 1,048,576), AUTO schedule."""
    cells = synth.field_cells(big, 16384, seed=1005)
    g = run_gpu(big, cells, 5e-9)
    assert (g["status"] == 0).all()
    costly = np.argsort(g["n_acc"] + g["n_rej"])[-16:]
    idx = np.unique(np.concatenate([synth.sample_indices(78, cells.n, 48), costly]))
    o = run_oracle(big, synth.subset(cells, idx), 5e-9)
    assert_parity(dict(T=g["T"][idx], Y=g["Y"][:, idx], status=g["status"][idx]), o)


def test_large_set_arrhenius_reaches_the_block_kernel(big, big_cells):
    """ln A and E changed through the C ABI equal the oracle run on the edited mechanism text."""
    import copy
    library()
    cells = synth.subset(big_cells, np.arange(48))
    edited = copy.deepcopy(big)
    changed = [0, 5, 77, 300] + [i for i, r in enumerate(big.reactions) if r.kind == "TROE"][:2]
    for r in changed:
        edited.reactions[r].A *= 2.0
        edited.reactions[r].E += 3.0          # kJ/mol
    m = rde_chem.Mechanism(big.to_text())
    lnA, E = rde_chem.rde_mech_get_arrhenius(m.handle, m.R)
    lnA, E = lnA.copy(), E.copy()
    lnA[changed] += np.log(2.0)
    E[changed] += 3000.0
    rde_chem.rde_mech_set_arrhenius(m.handle, lnA, E)
    p, T, Y = to_dev(cells.p), to_dev(cells.T), to_dev(cells.Y)
    st = torch.full((cells.n,), -1, dtype=torch.int32, device="cuda")
    rde_chem.rde_chem_advance_ex(m.handle, 5e-9, cells=rde_chem.make_block(p, T, Y, status=st))
    torch.cuda.synchronize()
    g = dict(T=T.cpu().numpy(), Y=Y.cpu().numpy(), status=st.cpu().numpy())
    m.close()
    o = run_oracle(edited, cells, 5e-9)
    assert_parity(g, o)
    base = run_oracle(big, cells, 5e-9)
    assert np.abs(base["T"] - o["T"]).max() > 1e-3     # the edit matters at this tolerance
