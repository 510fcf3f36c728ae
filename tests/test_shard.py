"""Multi-rank partitioning on CPU: two gloo ranks partition a cell field by the
per-cell cost of the previous step, advance their own cells with the oracle, and
agree through all-gather / max-reduce collectives on the control path only."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2508_16105_gb300 import shard, synth


def test_even_and_weighted_ranges():
    assert shard.even_ranges(10, 3) == [(0, 4), (4, 7), (7, 10)]
    cost = np.array([1, 1, 1, 1, 100, 1, 1, 1], float)
    r = shard.cost_weighted_ranges(cost, 2)
    assert r[0][0] == 0 and r[-1][1] == 8 and r[0][1] == r[1][0]
    loads = [cost[a:b].sum() for a, b in r]
    assert max(loads) <= 100 + 4
    u = synth.uniform(1, "cost", 100000) * 50 + 1
    r = shard.cost_weighted_ranges(u, 8)
    loads = [u[a:b].sum() for a, b in r]
    assert shard.imbalance(loads) < 1e-3
    assert sum(b - a for a, b in r) == 100000
    assert shard.cost_weighted_ranges(np.zeros(5), 2) == shard.even_ranges(5, 2)
    # the crossing cell goes to whichever side leaves the loads nearer even
    assert shard.cost_weighted_ranges(np.array([2, 2, 2, 10, 1, 1], float), 2) == [(0, 3), (3, 6)]
    assert shard.cost_weighted_ranges(np.array([1, 1, 10, 2, 2, 2], float), 2) == [(0, 3), (3, 6)]
    # two ranks: the cut is the best contiguous one (brute force over every cut)
    for s in range(20):
        c = synth.uniform(100 + s, "cost", 17) ** 3 * 10 + 0.01
        (a, b), _ = shard.cost_weighted_ranges(c, 2)
        best = min(max(c[:k].sum(), c[k:].sum()) for k in range(18))
        assert max(c[:b].sum(), c[b:].sum()) <= best * (1 + 1e-12)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch
    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mech = synth.h2_air_mechanism(16105)
    field = synth.field_cells(mech, 64, seed=1002)
    o = oracle.Oracle(mech.to_text())
    # step 1: even split; every rank learns all per-cell costs (control path)
    lo, hi = shard.even_ranges(field.n, world)[rank]
    sub = synth.subset(field, np.arange(lo, hi))
    T, Y, st, na, nr, _ = o.advance(sub.p, sub.T, sub.Y, 5e-9)
    mine = torch.tensor((na + nr).astype(np.float64))
    parts = [torch.zeros(b - a, dtype=torch.float64) for a, b in shard.even_ranges(field.n, world)]
    dist.all_gather(parts, mine)
    cost = torch.cat(parts).numpy()
    # step 2: cost-weighted split from the measured costs
    lo2, hi2 = shard.cost_weighted_ranges(cost, world)[rank]
    load = torch.tensor([cost[lo2:hi2].sum()], dtype=torch.float64)
    loads = [torch.zeros(1, dtype=torch.float64) for _ in range(world)]
    dist.all_gather(loads, load)
    tmax = torch.tensor([float(hi2 - lo2)])
    dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
    if rank == 0:
        out.put((cost.tolist(), [float(x) for x in loads], [shard.cost_weighted_ranges(cost, world)], float(tmax)))
    dist.destroy_process_group()


def _worker_measured(rank, world, port, out):
    """Ranks advance their cells with the oracle, take each cell's measured wall time as
    its cost (the counterpart of the library's per-cell clock cycles), and repartition
    through shard.repartition (an all-gather of the costs only)."""
    import time
    import torch
    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mech = synth.h2_air_mechanism(16105)
    field = synth.field_cells(mech, 40, seed=1002)
    o = oracle.Oracle(mech.to_text())
    ranges = shard.even_ranges(field.n, world)
    lo, hi = ranges[rank]
    cost = []
    for i in range(lo, hi):
        sub = synth.subset(field, np.array([i]))
        t0 = time.perf_counter()
        o.advance(sub.p, sub.T, sub.Y, 5e-9, threads=1)
        cost.append(time.perf_counter() - t0)
    new, loads, imb = shard.repartition(torch.tensor(cost), ranges, world)
    full = shard.gather_costs(torch.tensor(cost), ranges).numpy()
    if rank == 0:
        out.put((new, loads, imb, full.tolist()))
    dist.destroy_process_group()


def test_two_gloo_ranks_repartition_by_measured_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker_measured, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    new, loads, imb, full = q.get(timeout=300)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    full = np.array(full)
    assert len(full) == 40 and (full > 0).all()
    assert new == shard.cost_weighted_ranges(full, 2)
    assert new[0][0] == 0 and new[0][1] == new[1][0] and new[1][1] == 40
    after = [full[a:b].sum() for a, b in new]
    assert shard.imbalance(after) <= imb + 1e-12
    assert abs(sum(loads) - full.sum()) <= 1e-12 * full.sum()


def test_two_gloo_ranks_cost_weighted():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    cost, loads, ranges, tmax = q.get(timeout=300)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    cost = np.array(cost)
    even = [cost[a:b].sum() for a, b in shard.even_ranges(len(cost), 2)]
    assert shard.imbalance(loads) <= shard.imbalance(even) + 1e-12
    (r0, r1), = ranges
    assert r0[0] == 0 and r0[1] == r1[0] and r1[1] == len(cost)
    assert tmax == max(b - a for a, b in (r0, r1))
