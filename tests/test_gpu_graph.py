"""CUDA graphs and AMR-like block batching over consecutive steps.

- A library-captured graph of 5 steps equals 5 eager calls bit for bit (state
  and h_hint carried from step to step).
- A user-side torch.cuda.graph capture of the same call replays identically.
- Eight blocks of log-uniform sizes, each an RDE-like field mix, advanced in one
  launch per step through a device block table over 6 carried-forward steps,
  match the oracle carried forward the same way.
"""
import numpy as np
import pytest
import torch

from gpu_util import assert_parity, library, run_oracle, to_dev
from paper_2508_16105_gb300 import rde_chem, synth

pytestmark = pytest.mark.gpu


def _state(cells):
    return dict(p=to_dev(cells.p), T=to_dev(cells.T), Y=to_dev(cells.Y),
                h_hint=torch.zeros(cells.n, dtype=torch.float64, device="cuda"),
                status=torch.full((cells.n,), -1, dtype=torch.int32, device="cuda"))


def _blk(s):
    return rde_chem.make_block(s["p"], s["T"], s["Y"], h_hint=s["h_hint"], status=s["status"])


def test_graph_equals_eager():
    library()
    mech = synth.h2_air_mechanism(16105)
    cells = synth.field_cells(mech, 2000, seed=1002)
    m = rde_chem.Mechanism(mech.to_text())
    a, b = _state(cells), _state(cells)
    for _ in range(5):
        rde_chem.rde_chem_advance_ex(m.handle, 5e-9, cells=_blk(a))
    g = rde_chem.rde_chem_graph_create(m.handle, 5, 5e-9, cells=_blk(b))
    rde_chem.rde_chem_graph_launch(g)
    torch.cuda.synchronize()
    for k in ("T", "Y", "h_hint", "status"):
        assert torch.equal(a[k], b[k]), k
    rde_chem.rde_chem_graph_destroy(g)
    # a user-side torch graph capture of the same call
    c = _state(cells)
    blk = _blk(c)
    s = torch.cuda.Stream()
    rde_chem.rde_chem_advance_ex(m.handle, 5e-9, cells=blk, stream=s)   # warm-up outside capture
    torch.cuda.synchronize()
    c2 = _state(cells)
    for k in ("T", "Y", "h_hint"):
        c[k].copy_(c2[k])
    tg = torch.cuda.CUDAGraph()
    with torch.cuda.graph(tg, stream=s):
        rde_chem.rde_chem_advance_ex(m.handle, 5e-9, cells=blk, stream=s)
    for _ in range(5):
        tg.replay()
    torch.cuda.synchronize()
    for k in ("T", "Y", "h_hint"):
        assert torch.equal(a[k], c[k]), k
    m.close()


def test_amr_blocks_carried_forward():
    library()
    mech = synth.h2_air_mechanism(16105)
    sizes = synth.block_sizes(seed=1003, nblocks=8, lo=50, hi=1500)
    blocks_cells = [synth.field_cells(mech, int(n), seed=2000 + i) for i, n in enumerate(sizes)]
    states = [_state(c) for c in blocks_cells]
    table = rde_chem.BlockTable(states)
    m = rde_chem.Mechanism(mech.to_text())
    steps = 6
    g = rde_chem.rde_chem_graph_create(m.handle, steps, 5e-9, **table.call_args())
    rde_chem.rde_chem_graph_launch(g)
    torch.cuda.synchronize()
    rde_chem.rde_chem_graph_destroy(g)
    for i, (c, s) in enumerate(zip(blocks_cells, states)):
        idx = synth.sample_indices(10 + i, c.n, 40)
        sub = synth.subset(c, idx)
        T, Y, hint = sub.T, sub.Y, np.zeros(sub.n)
        for _ in range(steps):
            o = run_oracle(mech, synth.CellState(sub.p, T, Y, sub.cls), 5e-9, hint=hint)
            T, Y, hint = o["T"], o["Y"], o["hint"]
        gpu = dict(T=s["T"].cpu().numpy()[idx], Y=s["Y"].cpu().numpy()[:, idx], status=s["status"].cpu().numpy()[idx])
        assert_parity(gpu, o)
    m.close()
