"""Helpers shared by the GPU tests: run the CUDA path and the oracle on the same cells."""
import numpy as np
import torch

import oracle
from paper_2508_16105_gb300 import build, rde_chem, synth

T_REL_TOL = 1e-6     # |dT| / T
Y_ABS_TOL = 1e-9     # |dY_k|


def library():
    build.build_library()
    return rde_chem.load_library()


def to_dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def run_gpu(mech, cells, dt, rtol=1e-8, atol=1e-12, schedule=rde_chem.RDE_SCHED_QUEUE, hint=None,
            max_substeps=100000, ctas_per_sm=0, method=rde_chem.RDE_METHOD_RODAS3, flags=0, threads=0):
    library()
    m = rde_chem.Mechanism(mech.to_text() if hasattr(mech, "to_text") else mech, rtol, atol, max_substeps,
                           flags=flags, method=method)
    n = cells.n
    p, T, Y = to_dev(cells.p), to_dev(cells.T), to_dev(cells.Y)
    st = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    na = torch.zeros(n, dtype=torch.int32, device="cuda")
    nr = torch.zeros(n, dtype=torch.int32, device="cuda")
    hh = to_dev(hint) if hint is not None else None
    blk = rde_chem.make_block(p, T, Y, h_hint=hh, status=st, n_acc=na, n_rej=nr, n=n, ldY=n)
    rde_chem.rde_chem_advance_ex(m.handle, dt, cells=blk, schedule=schedule, ctas_per_sm=ctas_per_sm,
                                 threads_per_cta=threads)
    stats = rde_chem.rde_chem_get_stats(m.handle)
    torch.cuda.synchronize()
    out = dict(T=T.cpu().numpy(), Y=Y.cpu().numpy(), status=st.cpu().numpy(), n_acc=na.cpu().numpy(),
               n_rej=nr.cpu().numpy(), stats=stats, hint=hh.cpu().numpy() if hh is not None else None)
    m.close()
    return out


def run_oracle(mech, cells, dt, rtol=1e-8, atol=1e-12, hint=None, max_substeps=100000, threads=None,
               method=oracle.METHOD_RODAS3):
    import os
    o = oracle.Oracle(mech.to_text() if hasattr(mech, "to_text") else mech)
    T, Y, st, na, nr, hh = o.advance(cells.p, cells.T, cells.Y, dt,
                                     oracle.default_opts(rtol=rtol, atol=atol, max_substeps=max_substeps,
                                                         method=method),
                                     hint=hint, threads=threads or os.cpu_count())
    return dict(T=T, Y=Y, status=st, n_acc=na, n_rej=nr, hint=hh)


def assert_parity(g, o, T_tol=T_REL_TOL, Y_tol=Y_ABS_TOL):
    """Element-wise parity; cells reported BAD_STATE must be bitwise untouched on both sides."""
    assert np.array_equal(g["status"], o["status"]), (np.bincount(g["status"]), np.bincount(o["status"]))
    bad = g["status"] == 3
    assert np.array_equal(g["T"][bad], o["T"][bad], equal_nan=True)
    assert np.array_equal(g["Y"][:, bad], o["Y"][:, bad], equal_nan=True)
    ok = ~bad
    if not ok.any():
        return 0.0, 0.0
    dT = np.abs(g["T"][ok] - o["T"][ok]) / np.abs(o["T"][ok])
    dY = np.abs(g["Y"][:, ok] - o["Y"][:, ok])
    assert dT.max() <= T_tol, ("T", dT.max(), int(dT.argmax()))
    assert dY.max() <= Y_tol, ("Y", dY.max(), np.unravel_index(dY.argmax(), dY.shape))
    return dT.max(), dY.max()


SMALL_CASES = ["isomer_rev", "dimer", "robertson", "dissociation", "two_range", "troe"]


def small_case(name, n=64):
    """A small mechanism with a state and dt that exercise one feature (64 cells, T spread 2%)."""
    RU = 8.31446261815324
    if name == "isomer_rev":
        mech = synth.isomer_mechanism(reversible=True, A=5e5, b=0.3, E=10.0)
        Y = np.array([[0.7], [0.0], [0.3]])
        p, T, dt = 1e5, 1200.0, 1e-5
    elif name == "dimer":
        mech = synth.dimer_mechanism()
        Y = np.array([[0.9], [0.1]])
        p, T, dt = 2e5, 900.0, 1e-5
    elif name == "robertson":
        mech = synth.robertson_mechanism()
        Y = np.array([[1.0], [0.0], [0.0]])
        p, T, dt = RU * 1000.0, 1000.0, 40.0
    elif name == "dissociation":
        mech = synth.dissociation_mechanism()
        Y = np.array([[0.25], [0.0], [0.75]])
        p, T, dt = 101325.0, 4200.0, 1e-3
    elif name == "two_range":
        mech = synth.two_range_mechanism()
        Y = np.array([[0.8], [0.2]])
        p, T, dt = 1e5, 999.0, 1e-2
    else:
        mech = synth.isomer_mechanism(kind="TROE", reversible=True, A=3e5, b=0.3, E=40.0,
                                      low=(4e12, -0.5, 10.0), troe=(0.4, 300.0, 1800.0, 5000.0))
        mech.reactions[0].eff = {"X2": 2.0, "A": 0.7}
        Y = np.array([[0.5], [0.2], [0.3]])
        p, T, dt = 1e5, 1300.0, 1e-5
    cells = synth.CellState(np.full(n, p), np.full(n, T) * np.linspace(0.98, 1.02, n),
                            np.repeat(Y, n, axis=1), np.zeros(n, np.int8))
    return mech, cells, dt
