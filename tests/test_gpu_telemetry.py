"""Per-cell measured cost (rde_block.cycles): every processed cell gets the SM clock
cycles its integration took, and that cost tracks the cell's attempt count, for the
thread-per-cell kernel (queue and plain schedules, one block or a block table) and
the CTA-per-cell kernel.  The time-weighted shard planner partitions on it."""
import numpy as np
import pytest
import torch

from gpu_util import library, to_dev
from paper_2508_16105_gb300 import rde_chem, shard, synth

pytestmark = pytest.mark.gpu


def _rank_corr(a, b):
    ra = np.argsort(np.argsort(a)).astype(float)
    rb = np.argsort(np.argsort(b)).astype(float)
    return float(np.corrcoef(ra, rb)[0, 1])


@pytest.mark.parametrize("schedule", [rde_chem.RDE_SCHED_QUEUE, rde_chem.RDE_SCHED_PLAIN, rde_chem.RDE_SCHED_BLOCK])
def test_cycles_track_attempts(h2mech, schedule):
    library()
    n = 6000 if schedule != rde_chem.RDE_SCHED_BLOCK else 1500
    cells = synth.field_cells(h2mech, n, seed=1002)
    m = rde_chem.Mechanism(h2mech.to_text())
    p, T, Y = to_dev(cells.p), to_dev(cells.T), to_dev(cells.Y)
    na = torch.zeros(n, dtype=torch.int32, device="cuda")
    nr = torch.zeros(n, dtype=torch.int32, device="cuda")
    cyc = torch.full((n,), -1, dtype=torch.int64, device="cuda")
    rde_chem.rde_chem_advance_ex(m.handle, 5e-9, cells=rde_chem.make_block(p, T, Y, n_acc=na, n_rej=nr, cycles=cyc),
                                 schedule=schedule)
    torch.cuda.synchronize()
    m.close()
    c = cyc.cpu().numpy()
    att = (na + nr).cpu().numpy()
    assert (c > 0).all()
    assert _rank_corr(c, att) > 0.9, _rank_corr(c, att)
    # a partition by measured cost balances the attempts better than an even split
    ranges = shard.cost_weighted_ranges(c, 4)
    even = shard.even_ranges(n, 4)
    assert shard.imbalance([att[a:b].sum() for a, b in ranges]) <= shard.imbalance(
        [att[a:b].sum() for a, b in even]) + 0.05


def test_cycles_in_block_table(h2mech):
    library()
    cells = synth.field_cells(h2mech, 3000, seed=1002)
    m = rde_chem.Mechanism(h2mech.to_text())
    p, T, Y = to_dev(cells.p), to_dev(cells.T), to_dev(cells.Y)
    na = torch.zeros(cells.n, dtype=torch.int32, device="cuda")
    cyc = torch.zeros(cells.n, dtype=torch.int64, device="cuda")
    parts = [dict(p=p[a:b], T=T[a:b], Y=Y[:, a:b], n_acc=na[a:b], cycles=cyc[a:b]) for a, b in ((0, 1000), (1000, 3000))]
    table = rde_chem.BlockTable(parts)
    rde_chem.rde_chem_advance_ex(m.handle, 5e-9, **table.call_args())
    torch.cuda.synchronize()
    m.close()
    c = cyc.cpu().numpy()
    assert (c > 0).all()
    assert _rank_corr(c, na.cpu().numpy()) > 0.9
