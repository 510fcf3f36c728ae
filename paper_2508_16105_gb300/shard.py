"""Partitioning cells across ranks (one process per GPU).

Cells are independent during the chemistry step, so ranks exchange no data
while they advance; partitioning only decides which cells each rank owns.

The paper balances its CPU ranks on measured compute time ("cpuLoad") rather
than cell count (Section 3.3.1, Table 12), because chemistry cost concentrates
where combustion occurs (Section 1).  ``cost_weighted_ranges`` is that rule for
contiguous cell ranges: given each cell's cost from the previous step (its
accepted + rejected substep count, which the library reports per cell), it cuts
the range so every rank gets close to the same total cost.  ``imbalance`` is
the paper's trigger quantity (max load / mean load - 1; it redistributes when
this exceeds 0.1).
"""
from __future__ import annotations

import numpy as np


def even_ranges(n: int, world: int) -> list:
    """Contiguous [lo, hi) ranges of n cells, sizes differing by at most one."""
    base, extra = divmod(n, world)
    out, lo = [], 0
    for r in range(world):
        hi = lo + base + (1 if r < extra else 0)
        out.append((lo, hi))
        lo = hi
    return out


def cost_weighted_ranges(cost: np.ndarray, world: int) -> list:
    """Contiguous ranges whose summed cost is as even as prefix cuts allow.

    Rank r's range ends next to the cell whose cost carries the prefix across
    (r+1)/world of the total: before or after that cell, whichever leaves the
    prefix nearer the target (for two ranks this is the best contiguous cut).
    Every cell belongs to exactly one range.
    """
    cost = np.asarray(cost, dtype=np.float64)
    n = cost.shape[0]
    if n == 0:
        return [(0, 0)] * world
    if np.any(cost < 0):
        raise ValueError("cost must be non-negative")
    total = float(cost.sum())
    if total == 0.0:
        return even_ranges(n, world)
    prefix = np.cumsum(cost)
    cuts = [0]
    for r in range(1, world):
        target = total * r / world
        i = int(np.searchsorted(prefix, target, side="left"))   # first cell whose prefix reaches the target
        c = i + 1
        if i < n and i > 0 and target - prefix[i - 1] < prefix[i] - target:
            c = i   # the crossing cell goes to the next rank
        cuts.append(min(max(c, cuts[-1]), n))
    cuts.append(n)
    return [(cuts[r], cuts[r + 1]) for r in range(world)]


def imbalance(loads) -> float:
    """max(load) / mean(load) - 1 (0 for a perfectly balanced partition)."""
    loads = np.asarray(loads, dtype=np.float64)
    m = loads.mean()
    return float(loads.max() / m - 1.0) if m > 0 else 0.0


def gather_costs(local_cost, ranges, group=None):
    """The whole field's per-cell cost on every rank, from each rank's cost of its own
    range (ranges[r] = (lo, hi) of rank r; local_cost holds hi - lo values).

    torch.distributed must be initialised (NCCL for CUDA tensors, gloo for CPU
    ones); only these cost values cross ranks.  Returns a float64 tensor on
    local_cost's device."""
    import torch
    import torch.distributed as dist
    local = torch.as_tensor(local_cost).to(torch.float64)
    width = max(b - a for a, b in ranges)
    buf = torch.zeros(width, dtype=torch.float64, device=local.device)
    buf[: local.numel()] = local
    parts = [torch.empty(width, dtype=torch.float64, device=local.device) for _ in ranges]
    dist.all_gather(parts, buf, group=group)
    return torch.cat([part[: b - a] for part, (a, b) in zip(parts, ranges)])


def repartition(local_cost, ranges, world: int, group=None):
    """Next step's contiguous ranges from this step's measured per-cell costs:
    (new ranges, per-rank loads under the old ranges, imbalance of the old ones)."""
    cost = gather_costs(local_cost, ranges, group).cpu().numpy()
    loads = [float(cost[a:b].sum()) for a, b in ranges]
    return cost_weighted_ranges(cost, world), loads, imbalance(loads)

