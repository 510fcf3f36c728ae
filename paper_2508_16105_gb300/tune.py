"""Autotuner for the chemistry step's launch configuration.

The tunable choices are the threads per cell (one thread per cell with its
matrix in shared-memory lane slots, or 128 threads per cell in the CTA-per-cell
kernel), the schedule of the thread-per-cell kernel (plain one-pass or
persistent queue) and, where the shared-memory footprint lets more than one
CTA share an SM, the number of persistent CTAs per SM.  Each candidate advances the same seeded sample of the caller's cells once
(from a fresh copy of the state) and is timed with CUDA events; the fastest is
cached on disk, keyed by the mechanism text's hash, the GPU name, the species
count and the log2 bucket of the cell count.  The cache file is
$RDE_TUNE_CACHE, default ~/.cache/rde_chem_tune.json.

The sample holds at least two cells per thread-per-cell lane of the GPU (SMs x
threads per CTA x CTAs per SM, times two) when the caller has that many: a
smaller sample leaves SMs idle under one thread per cell while the CTA-per-cell
kernel still spreads its few cells over every SM, and so favours the latter for
a workload whose full size would fill the GPU either way.
"""
from __future__ import annotations

import hashlib
import json
import math
import os

import torch

from . import rde_chem


def cache_path() -> str:
    return os.environ.get("RDE_TUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "rde_chem_tune.json"))


def _key(mech_text: str, K: int, n: int) -> str:
    h = hashlib.sha256(mech_text.encode()).hexdigest()[:16]
    dev = torch.cuda.get_device_name()
    return "%s|%s|K%d|n2^%d" % (h, dev, K, max(0, int(math.log2(max(n, 1)))))


def _load() -> dict:
    try:
        with open(cache_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(d: dict):
    path = cache_path()
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + ".%d.tmp" % os.getpid()
    with open(tmp, "w") as f:
        json.dump(d, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def candidates(max_ctas_per_sm: int, thread_per_cell: bool = True, wide: bool = False) -> list:
    """Launches to time: thread per cell (plain; queue with 128-thread CTAs at 1..max CTAs
    per SM; the wide 256-thread queue kernel where the handle has one) when a
    thread-per-cell kernel serves the mechanism, and the CTA-per-cell kernel (128
    threads per cell)."""
    out = []
    if thread_per_cell:
        out.append(dict(schedule=rde_chem.RDE_SCHED_PLAIN, ctas_per_sm=0, threads_per_cta=128))
        for c in range(1, max(1, max_ctas_per_sm) + 1):
            out.append(dict(schedule=rde_chem.RDE_SCHED_QUEUE, ctas_per_sm=c, threads_per_cta=128))
        if wide:
            out.append(dict(schedule=rde_chem.RDE_SCHED_QUEUE, ctas_per_sm=0, threads_per_cta=256))
    out.append(dict(schedule=rde_chem.RDE_SCHED_BLOCK, ctas_per_sm=0, threads_per_cta=0))
    return out


def tune(mech: "rde_chem.Mechanism", mech_text: str, p, T, Y, dt: float, sample: int = 16384,
         use_cache: bool = True) -> dict:
    """Best launch configuration for advancing cells like (p, T, Y) over dt.

    p, T: [n] and Y: [K, n] device tensors (not modified).  Returns a dict with
    schedule, ctas_per_sm, the measured milliseconds of every candidate and
    whether it came from the cache.
    """
    n = int(T.shape[0])
    key = _key(mech_text, mech.K, n)
    cache = _load() if use_cache else {}
    if key in cache:
        r = dict(cache[key])
        r["cached"] = True
        return r
    info = rde_chem.rde_chem_kernel_info(mech.handle)
    lanes = torch.cuda.get_device_properties(T.device).multi_processor_count * info["threads_per_cta"] * \
        max(1, info["max_ctas_per_sm"])
    m = min(n, max(sample, 2 * lanes))
    idx = torch.arange(m, device=T.device) * max(1, n // m)
    ps, Ts, Ys = p[idx].contiguous(), T[idx].contiguous(), Y[:, idx].contiguous()
    variant, _ = rde_chem.rde_chem_kernel_variant(mech.handle)
    results = []
    # the wide 256-thread queue kernel is a candidate where the handle can build it (its
    # first call compiles it, outside the timing)
    wide = variant == rde_chem.RDE_KERNEL_SPECIALIZED
    if wide:
        try:
            blk = rde_chem.make_block(ps[:1], Ts[:1].clone(), Ys[:, :1].clone())
            rde_chem.rde_chem_advance_ex(mech.handle, dt, cells=blk, threads_per_cta=256)
            torch.cuda.synchronize()
        except rde_chem.RdeError:
            wide = False
    for cand in candidates(info["max_ctas_per_sm"], variant != rde_chem.RDE_KERNEL_BLOCK, wide):
        Tw, Yw = Ts.clone(), Ys.clone()
        blk = rde_chem.make_block(ps, Tw, Yw, n=m, ldY=m)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        rde_chem.rde_chem_advance_ex(mech.handle, dt, cells=blk, **cand)
        b.record()
        torch.cuda.synchronize()
        results.append(dict(cand, ms=a.elapsed_time(b)))
    best = min(results, key=lambda r: r["ms"])
    out = dict(schedule=best["schedule"], ctas_per_sm=best["ctas_per_sm"], threads_per_cta=best["threads_per_cta"],
               trials=results, sample=m)
    if use_cache:
        cache[key] = out
        _store(cache)
    out = dict(out)
    out["cached"] = False
    return out
