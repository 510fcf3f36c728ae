"""Benchmark of the per-cell FP64 chemistry step on GB300.

Workload (default): the batched, uneven RDE-like 2D field: 2,097,152 cells of
the seeded 9-species / 21-reaction H2-air mechanism (90 % fresh reactants at
300-600 K, 5 % post-shock front at 1500-3500 K and 1-3 MPa, 5 % burnt products),
dt = 5e-9 s, rtol 1e-8 / atol 1e-12, advanced by the persistent queue kernel in
one launch per step.  A step restores the field's initial state (device copy)
and advances every cell over dt; the metric is cell-chemistry steps per second.

Prints one JSON line (rank 0).  ``--impl reference`` times the CPU oracle on the
host cores instead, each step a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "cell-chemistry steps/s (FP64, H2-air) and adjoint/forward time ratio"
UNIT = "cell-steps/s"
FIELD_CELLS = 2097152
DT = 5e-9
MECH_SEED = 16105
FIELD_SEED = 1002
CPU_SAMPLE = 16384          # cells of the field timed on the host for cpu_baseline
REF_SAMPLE = 4096           # cells per step of the --impl reference arm

# DRAM traffic per cell-step of the queue kernel from one ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum of the timed launch on the
# 2,097,152-cell field, queue in cell-index order, divided by its cells), keyed by the
# hash of the kernel sources it was measured on and the kernel ("/w": the wide
# 256-thread queue kernel, profiles/rde_jit_queue_w_field2M.md; "/n": the 128-thread
# one): a changed kernel reports null.
TRAFFIC_BYTES_PER_CELL = {"00d40b2396d7f410/w": (268556032.0 + 15547633920.0) / 2097152}
# Executed FP64 flops per attempt of the specialised queue kernel, 2 dfma + dadd + dmul
# thread instructions of one ncu-captured launch on the 2,097,152-cell field divided by
# its attempts (the same profile), keyed like the traffic above.
EXECUTED_FLOPS_PER_ATTEMPT = {"00d40b2396d7f410/w": (2 * 1857192399372 + 673102120819 + 426789399575) / 587906652}
KERNEL_SOURCES = ["chem_device.cuh", "chem_kernel_body.cuh", "chem_kernels.cu", "jit.cu", "fastmath.cuh",
                  "fastmath_tables.h", "mech_layout.h"]


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2508_16105_gb300", "csrc")
    for name in KERNEL_SOURCES:
        with open(os.path.join(d, name), "rb") as f:
            h.update(name.encode() + f.read())
    return h.hexdigest()[:16]


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid: str | None):
        self.proc = None
        self.uuid = uuid

    def start(self):
        cmd = ["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits", "-lms", "200"]
        if self.uuid:
            cmd.insert(1, "--id=" + self.uuid)
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self) -> dict | None:
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        rows = []
        for line in out.strip().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                rows.append((float(parts[0]), float(parts[1]), float(parts[2]), parts[3:]))
            except ValueError:
                continue
        if not rows:
            return None
        load = [r for r in rows if r[2] > 0.3 * max(x[2] for x in rows)] or rows
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in load for i, v in enumerate(r[3][1:5]) if v.lower() == "active"})
        return {"sm_mhz": float(np.median([r[0] for r in load])), "sm_max_mhz": max(r[1] for r in rows),
                "power_w_max": max(r[2] for r in rows), "samples": len(load), "reasons": reasons}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def reference_arm(args, world, rank):
    """CPU oracle on the host cores, each step a bounded sample of the field."""
    if rank != 0:
        return 0
    import oracle
    from paper_2508_16105_gb300 import synth
    mech = synth.h2_air_mechanism(MECH_SEED)
    field = synth.field_cells(mech, FIELD_CELLS, seed=FIELD_SEED)
    o = oracle.Oracle(mech.to_text())
    cores = os.cpu_count() or 1
    times = []
    for s in range(args.warmup + args.steps):
        idx = synth.sample_indices(500 + s, field.n, REF_SAMPLE)
        sub = synth.subset(field, idx)
        t0 = time.perf_counter()
        o.advance(sub.p, sub.T, sub.Y, DT, threads=cores)
        times.append(time.perf_counter() - t0)
    t = sum(times[args.warmup:])
    value = REF_SAMPLE * args.steps / t
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "gpu_launches": 0,
            "config": {"workload": "rde_field_2d_h2air_9sp21rx_dt5e-9",
                       "cells": FIELD_CELLS, "sample_cells_per_step": REF_SAMPLE},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "%d cells per step drawn from the %d-cell field" % (REF_SAMPLE, FIELD_CELLS)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def cpu_baseline(mech, field, sample: int) -> dict:
    import oracle
    from paper_2508_16105_gb300 import synth
    o = oracle.Oracle(mech.to_text())
    cores = os.cpu_count() or 1
    idx = synth.sample_indices(99, field.n, sample)
    sub = synth.subset(field, idx)
    t0 = time.perf_counter()
    o.advance(sub.p, sub.T, sub.Y, DT, threads=cores)
    t = time.perf_counter() - t0
    return {"value": sample / t, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "%d cells drawn uniformly from the %d-cell field, one dt each, %.1f s wall on %d threads"
                      % (sample, field.n, t, cores)}


AMR_BLOCKS = 64
AMR_SEED = 1003


def amr_graph_leg(nsteps: int = 100, warmup: int = 1, curve: bool = True, scale_cells: int | None = None,
                  threads: int = 0) -> dict:
    """64 AMR-like blocks (log-uniform 1e4..5e5 cells, each an RDE-like field mix) in one
    block table, ``nsteps`` consecutive dt = 5e-9 s steps with T, Y and h_hint carried
    forward, replayed as one CUDA graph.  Value: cell-steps per second over the steps.
    With ``curve`` the same steps are also run eagerly from the same start and each is
    timed (the per-step cost falls as the carried step sizes and the chemistry relax).
    ``threads``: threads per CTA of the queue kernel (0/128, or 256 for the wide one)."""
    import torch
    from paper_2508_16105_gb300 import rde_chem, synth

    mech = synth.h2_air_mechanism(MECH_SEED)
    sizes = synth.block_sizes(seed=AMR_SEED, nblocks=AMR_BLOCKS, lo=1e4, hi=5e5)
    if scale_cells:                   # scaled-down variant for quick runs
        sizes = np.maximum(1, (sizes * (scale_cells / sizes.sum())).astype(np.int64))
    cells = [synth.field_cells(mech, int(n), seed=3000 + i) for i, n in enumerate(sizes)]
    n_total = int(sizes.sum())
    init = [dict(p=torch.as_tensor(c.p, device="cuda"), T=torch.as_tensor(c.T, device="cuda"),
                 Y=torch.as_tensor(np.ascontiguousarray(c.Y), device="cuda")) for c in cells]
    del cells
    work = [dict(p=b["p"], T=b["T"].clone(), Y=b["Y"].clone(),
                 h_hint=torch.zeros_like(b["T"])) for b in init]
    table = rde_chem.BlockTable(work)
    m = rde_chem.Mechanism(mech.to_text())

    def reset():
        for w, b in zip(work, init):
            w["T"].copy_(b["T"])
            w["Y"].copy_(b["Y"])
            w["h_hint"].zero_()

    call = dict(table.call_args(), threads_per_cta=threads)
    for _ in range(warmup):                           # warm-up: single steps, then reset
        rde_chem.rde_chem_advance_ex(m.handle, DT, **call)
    reset()
    g = rde_chem.rde_chem_graph_create(m.handle, nsteps, DT, **call)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    rde_chem.rde_chem_graph_launch(g)
    e1.record()
    torch.cuda.synchronize()
    t_graph = e0.elapsed_time(e1) / 1e3
    rde_chem.rde_chem_graph_destroy(g)
    out = {"workload": "amr_blocks_%d_graph%d_h2air_9sp21rx_dt5e-9" % (len(sizes), nsteps),
           "value": n_total * nsteps / t_graph, "unit": UNIT, "steps": nsteps, "graph_s": t_graph,
           "ms_per_step": 1e3 * t_graph / nsteps, "blocks": len(sizes), "cells": n_total,
           "block_min": int(sizes.min()), "block_max": int(sizes.max()), "graph": True,
           "sizes": "log-uniform in [1e4, 5e5] cells, seed %d: %d cells in all (the distribution's mean "
                    "gives 8.0 M; this draw gives %.2f M)" % (AMR_SEED, n_total, n_total / 1e6),
           "carried": "T, Y and h_hint carried from step to step; the step restarts the queue, not the state",
           "threads_per_cta": threads if threads else 128}
    if curve:
        reset()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(nsteps + 1)]
        ev[0].record()
        attempts = []
        for i in range(nsteps):
            rde_chem.rde_chem_advance_ex(m.handle, DT, **call)
            ev[i + 1].record()
            attempts.append(rde_chem.rde_chem_get_stats(m.handle))
        torch.cuda.synchronize()
        out["per_step_ms_eager"] = [round(ev[i].elapsed_time(ev[i + 1]), 3) for i in range(nsteps)]
        out["per_step_attempts_per_cell"] = [round((a["accepted"] + a["rejected"]) / n_total, 2) for a in attempts]
    m.close()
    del work, init, table
    torch.cuda.empty_cache()
    return out


def amr_graph_workload(args) -> int:
    from paper_2508_16105_gb300 import build, rde_chem
    build.build_library()
    rde_chem.load_library()
    leg = amr_graph_leg(args.amr_steps, args.warmup, args.curve,
                        None if args.cells == FIELD_CELLS else args.cells, args.threads)
    out = {"metric": METRIC, "value": leg["value"], "unit": UNIT, "n_gpus": 1, "steps": leg["steps"],
           "warmup": args.warmup, "ms_per_step": leg["ms_per_step"], "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "gpu_launches": leg["steps"],
           "config": {k: leg[k] for k in ("workload", "blocks", "cells", "block_min", "block_max", "graph",
                                          "sizes", "carried", "threads_per_cta")}, "amr": leg}
    print(json.dumps(out), flush=True)
    return 0


METHOD_CELLS = 65536        # field sample of the work-precision comparison
METHOD_RTOLS = (1e-4, 1e-6, 1e-8)


def methods_workload(args) -> int:
    """Work-precision of the three integrators (RODAS3, ROS2, and the order-3 linearly
    implicit Euler extrapolation) on a seeded 65,536-cell sample of the 2D field at
    dt = 5e-9 s: for each rtol (atol 1e-12) the kernel time of one step and the error
    against RODAS3 at rtol 1e-12 (max |dT|/T, max |dY|).
    Value: ROS2 time / RODAS3 time at rtol 1e-8 (lower favours ROS2)."""
    import torch
    from paper_2508_16105_gb300 import build, rde_chem, synth

    build.build_library()
    rde_chem.load_library()
    mech = synth.h2_air_mechanism(MECH_SEED)
    cells = synth.field_cells(mech, METHOD_CELLS, seed=FIELD_SEED)
    p = torch.as_tensor(cells.p, device="cuda")
    T0 = torch.as_tensor(cells.T, device="cuda")
    Y0 = torch.as_tensor(np.ascontiguousarray(cells.Y), device="cuda")
    text = mech.to_text()

    def run(method, rtol, reps=1):
        m = rde_chem.Mechanism(text, rtol=rtol, method=method)
        T, Y = T0.clone(), Y0.clone()
        rde_chem.rde_chem_advance(m.handle, cells.n, p, T, Y, DT)      # warm-up (and first-use set-up)
        ms = []
        for _ in range(reps):
            T.copy_(T0)
            Y.copy_(Y0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            rde_chem.rde_chem_advance(m.handle, cells.n, p, T, Y, DT)
            e1.record()
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        st = rde_chem.rde_chem_get_stats(m.handle)
        m.close()
        return T, Y, min(ms), st

    Tref, Yref, ms_ref, _ = run(rde_chem.RDE_METHOD_RODAS3, 1e-12)
    rows = []
    for rtol in METHOD_RTOLS:
        for name, meth in (("RODAS3", rde_chem.RDE_METHOD_RODAS3), ("ROS2", rde_chem.RDE_METHOD_ROS2),
                           ("EXTRAP3", rde_chem.RDE_METHOD_EXTRAP)):
            T, Y, ms, st = run(meth, rtol, reps=max(1, args.steps))
            rows.append({"method": name, "rtol": rtol, "kernel_ms": ms,
                         "attempts_per_cell": (st["accepted"] + st["rejected"]) / cells.n,
                         "max_rel_dT": float(((T - Tref).abs() / Tref).max()),
                         "max_abs_dY": float((Y - Yref).abs().max()), "failed": st["failed"]})
    t = {(r["method"], r["rtol"]): r["kernel_ms"] for r in rows}
    ratio = t[("ROS2", 1e-8)] / t[("RODAS3", 1e-8)]
    out = {"metric": "integrator work-precision, ROS2 / RODAS3 step time at rtol 1e-8", "value": ratio,
           "unit": "x", "n_gpus": 1, "steps": max(1, args.steps), "warmup": 1, "ms_per_step": t[("RODAS3", 1e-8)],
           "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "gpu_launches": len(rows) * max(1, args.steps),
           "config": {"workload": "methods_field_sample_%d_h2air_9sp21rx_dt5e-9" % cells.n, "cells": cells.n,
                      "reference": "RODAS3 at rtol 1e-12 (%.1f ms)" % ms_ref, "atol": 1e-12},
           "rows": rows}
    print(json.dumps(out), flush=True)
    return 0


LARGE_CELLS = 1048576       # 53-species stress field
LARGE_SAMPLE = 16384        # seeded 1/64 sample of it, timed and reported as a rate
LARGE_SEED = 1005


def large_field_leg(steps: int, warmup: int, sample: int = LARGE_SAMPLE) -> dict:
    """The 53-species / 325-reaction stress mechanism (20 three-body, 10 Troe) on the
    1,048,576-cell field mix: a seeded 1/64 sample of the cells is advanced over
    dt = 5e-9 s by the CTA-per-cell kernel (54 x 54 Jacobian and LU per cell).
    The rate (cell-steps/s) is that of the sample; the full field's step time is
    the cells divided by that rate."""
    import torch
    from paper_2508_16105_gb300 import rde_chem, roofline, synth
    mech = synth.large_mechanism(MECH_SEED)
    field = synth.field_cells(mech, LARGE_CELLS, seed=LARGE_SEED)
    idx = synth.sample_indices(LARGE_SEED, field.n, sample)
    cells = synth.subset(field, idx)
    del field
    n = cells.n
    m = rde_chem.Mechanism(mech.to_text())
    info = rde_chem.rde_chem_kernel_info(m.handle)
    p = torch.as_tensor(cells.p, device="cuda")
    T0 = torch.as_tensor(cells.T, device="cuda")
    Y0 = torch.as_tensor(np.ascontiguousarray(cells.Y), device="cuda")
    T, Y = T0.clone(), Y0.clone()
    blk = rde_chem.make_block(p, T, Y, n=n, ldY=n)
    stream = torch.cuda.current_stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * steps)]
    for _ in range(warmup):
        T.copy_(T0)
        Y.copy_(Y0)
        rde_chem.rde_chem_advance_ex(m.handle, DT, cells=blk, stream=stream)
    torch.cuda.synchronize()
    for i in range(steps):
        T.copy_(T0)
        Y.copy_(Y0)
        ev[2 * i].record(stream)
        rde_chem.rde_chem_advance_ex(m.handle, DT, cells=blk, stream=stream)
        ev[2 * i + 1].record(stream)
    torch.cuda.synchronize()
    stats = rde_chem.rde_chem_get_stats(m.handle)
    ks = float(np.mean([ev[2 * i].elapsed_time(ev[2 * i + 1]) / 1e3 for i in range(steps)]))
    attempts = stats["accepted"] + stats["rejected"]
    fl = roofline.flops_per_attempt(mech)["total"]
    flw = roofline.flops_per_attempt(mech, weighted=True)["total"]
    achieved = fl * attempts / ks / 1e9
    m.close()
    return {"workload": "stress_53sp325rx_field_1048576_sample%d_dt5e-9" % n, "species": mech.K,
            "reactions": mech.R, "cells_sampled": n, "cells_full": LARGE_CELLS, "kernel": "chem_large_kernel",
            "schedule": "block (CTA per cell, work queue)", "threads_per_cta": info["threads_per_cta"],
            "ctas_per_sm": info["max_ctas_per_sm"], "shared_bytes": info["shared_bytes"],
            "kernel_ms": 1e3 * ks, "value": n / ks, "unit": UNIT,
            "full_field_step_s": LARGE_CELLS * ks / n, "substeps_per_cell": attempts / n,
            "failed_cells": stats["failed"],
            "roofline": {"bound": "alu", "achieved": achieved, "peak": roofline.FP64_PEAK_GFLOPS,
                         "unit": "GFLOP/s", "frac": achieved / roofline.FP64_PEAK_GFLOPS,
                         "flops_per_attempt": fl, "attempts_per_launch": attempts,
                         "flop_rule": "exp, log, division and root = 1 flop; FMA = 2",
                         "weighted": {"flops_per_attempt": flw,
                                      "frac": flw * attempts / ks / 1e9 / roofline.FP64_PEAK_GFLOPS}}}


LARGE_ADJ_SAMPLE = 1216     # cells of the 53-species adjoint timing (8 per SM)


def large_adjoint_leg(sample: int = LARGE_ADJ_SAMPLE) -> dict:
    """The 53-species adjoint: a seeded sample of the stress field's cells, the CTA-per-
    cell forward step (with step counts) and the CTA-per-cell discrete adjoint (stage
    recompute) with seeded cotangents, each timed once with CUDA events."""
    import torch
    from paper_2508_16105_gb300 import rde_chem, synth
    mech = synth.large_mechanism(MECH_SEED)
    field = synth.field_cells(mech, LARGE_CELLS, seed=LARGE_SEED)
    cells = synth.subset(field, synth.sample_indices(LARGE_SEED + 1, field.n, sample))
    del field
    n = cells.n
    m = rde_chem.Mechanism(mech.to_text())
    p = torch.as_tensor(cells.p, device="cuda")
    T0 = torch.as_tensor(cells.T, device="cuda")
    Y0 = torch.as_tensor(np.ascontiguousarray(cells.Y), device="cuda")
    g = synth.normal(2005, "cot", (mech.K + 1) * n).reshape(mech.K + 1, n)
    gT = torch.as_tensor(g[mech.K] / np.abs(cells.T).max(), device="cuda")
    gY = torch.as_tensor(np.ascontiguousarray(g[:mech.K] / np.maximum(np.abs(cells.Y).max(axis=1, keepdims=True),
                                                                       1e-3)), device="cuda")
    T, Y = T0.clone(), Y0.clone()
    n_acc = torch.zeros(n, dtype=torch.int32, device="cuda")
    st = torch.zeros(n, dtype=torch.int32, device="cuda")
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    ev[0].record()
    rde_chem.rde_chem_advance_ex(m.handle, DT, cells=rde_chem.make_block(p, T, Y, n_acc=n_acc), threads_per_cta=128)
    ev[1].record()
    torch.cuda.synchronize()
    total = int(n_acc.sum().item())
    ws = torch.empty(rde_chem.rde_chem_adjoint_workspace_steps(m.handle, n, total), dtype=torch.uint8, device="cuda")
    gT0, gY0 = torch.empty_like(T0), torch.empty_like(Y0)
    glnA = torch.empty(mech.R, dtype=torch.float64, device="cuda")
    gE = torch.empty(mech.R, dtype=torch.float64, device="cuda")
    ev[2].record()
    rde_chem.rde_chem_advance_adjoint_ex(m.handle, DT, p, T0, Y0, n_acc, total, gT, gY, gT0, gY0, glnA, gE, ws,
                                      status=st)
    ev[3].record()
    torch.cuda.synchronize()
    t_f = ev[0].elapsed_time(ev[1]) / 1e3
    t_b = ev[2].elapsed_time(ev[3]) / 1e3
    out = {"cells": n, "forward_s": t_f, "adjoint_s": t_b, "ratio": t_b / t_f, "accepted_steps": total,
           "adjoint_cell_steps_per_s": n / t_b, "workspace_GB": ws.numel() / 1e9,
           "kernel": "chem_large_adjoint_kernel (CTA per cell, one per SM, stage recompute)",
           "failed_cells": int((st != 0).sum().item()),
           "grad_norms": {"gT0": float(gT0.norm()), "glnA": float(glnA.norm()), "gE": float(gE.norm())}}
    m.close()
    del ws
    torch.cuda.empty_cache()
    return out


def lu54_leg(batch: int = 65536, n: int = 54, reps: int = 3) -> dict:
    """Batched 54 x 54 LU with partial pivoting, trailing update on the FP64 tensor cores
    (DMMA) vs the CUDA cores (DFMA), same blocked algorithm otherwise; seeded matrices
    with a dominant diagonal (the shape of I/(gamma h) - J).  Algorithmic work 2n^3/3."""
    import torch
    from paper_2508_16105_gb300 import rde_chem, roofline, synth
    g = synth.normal(54, "lu54", n * n * 64).reshape(64, n, n)
    base = torch.tensor(g, device="cuda") + 50.0 * torch.eye(n, device="cuda", dtype=torch.float64)
    A0 = base.repeat((batch + 63) // 64, 1, 1)[:batch].contiguous()      # 1.5 GB at 65,536 matrices
    piv = torch.zeros((batch, n), dtype=torch.int32, device="cuda")
    A = torch.empty_like(A0)
    out = {"batch": batch, "n": n, "flops_per_lu": 2.0 * n ** 3 / 3.0}
    for name, dm in (("dfma", 0), ("dmma", 1)):
        ts = []
        for _ in range(reps + 1):
            A.copy_(A0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            rde_chem.rde_selftest_batched_lu(dm, A, piv)
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1) / 1e3)
        t = float(np.mean(ts[1:]))
        gf = out["flops_per_lu"] * batch / t / 1e9
        out[name] = {"ms": 1e3 * t, "gflops": gf, "frac": gf / roofline.FP64_PEAK_GFLOPS}
    out["dmma_over_dfma"] = out["dfma"]["ms"] / out["dmma"]["ms"]
    del A, A0
    torch.cuda.empty_cache()
    return out


ADJ_CELLS = 262144
ADJ_DT = 1e-8


def adjoint_leg(mech, n: int) -> dict:
    """Front-heavy field (50 % front, 25 % fresh, 25 % burnt), dt = 1e-8 s: time the forward
    step (with per-cell step counts) and the discrete adjoint with seeded cotangents, with
    stage recompute and, where the device holds their workspace, with stage checkpoints
    (the reported adjoint).  The first adjoint call, which builds the mechanism's adjoint
    kernels, is not timed."""
    import torch
    from paper_2508_16105_gb300 import rde_chem, synth
    cells = synth.field_cells(mech, n, seed=1004, fractions=(0.25, 0.50, 0.25))
    m = rde_chem.Mechanism(mech.to_text())
    p = torch.as_tensor(cells.p, device="cuda")
    T0 = torch.as_tensor(cells.T, device="cuda")
    Y0 = torch.as_tensor(np.ascontiguousarray(cells.Y), device="cuda")
    # cotangents ~ N(0, 1) scaled by 1/max|y| per component (species scale floored at 1e-3:
    # some radicals start at exactly zero in every cell)
    g = synth.normal(2001, "cot", (mech.K + 1) * n).reshape(mech.K + 1, n)
    gT = torch.as_tensor(g[mech.K] / np.abs(cells.T).max(), device="cuda")
    gY = torch.as_tensor(np.ascontiguousarray(g[:mech.K] / np.maximum(np.abs(cells.Y).max(axis=1, keepdims=True),
                                                                       1e-3)), device="cuda")
    n_acc = torch.zeros(n, dtype=torch.int32, device="cuda")
    T, Y = T0.clone(), Y0.clone()

    def fwd(threads=128):
        # 128 threads: the arithmetic the adjoint's re-integration retraces (its n_acc sizes
        # the recorded mode); 256: the fastest forward, for the second ratio
        T.copy_(T0)
        Y.copy_(Y0)
        rde_chem.rde_chem_advance_ex(m.handle, ADJ_DT, cells=rde_chem.make_block(p, T, Y, n_acc=n_acc),
                                     threads_per_cta=threads)

    wide_ok = True
    try:
        fwd(256)    # builds the wide kernel (untimed); its counts are replaced by the 128-thread pass
    except rde_chem.RdeError:
        wide_ok = False
    fwd()
    torch.cuda.synchronize()
    total = int(n_acc.sum().item())
    small = rde_chem.rde_chem_adjoint_workspace_steps(m.handle, n, total)
    big = rde_chem.rde_chem_adjoint_workspace_checkpointed(m.handle, n, total)
    # stage checkpoints when the device holds them with 16 GB to spare, else stage recompute
    torch.cuda.empty_cache()
    ws = None
    if big + (16 << 30) <= torch.cuda.mem_get_info()[0]:
        try:
            ws = torch.empty(big, dtype=torch.uint8, device="cuda")
        except torch.cuda.OutOfMemoryError:
            ws = None
    stages = ws is not None
    if ws is None:
        ws = torch.empty(small, dtype=torch.uint8, device="cuda")
    gT0, gY0 = torch.empty_like(T0), torch.empty_like(Y0)
    glnA = torch.empty(mech.R, dtype=torch.float64, device="cuda")
    gE = torch.empty(mech.R, dtype=torch.float64, device="cuda")

    def bwd(nbytes):
        rde_chem.rde_chem_advance_adjoint_ex(m.handle, ADJ_DT, p, T0, Y0, n_acc, total, gT, gY, gT0, gY0, glnA, gE,
                                          ws[:nbytes])

    bwd(small)      # first call: builds the mechanism's specialised adjoint kernels (load-time work, untimed)
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    ev[0].record()
    fwd()
    ev[1].record()
    bwd(small)                   # step checkpoints: the reverse sweep recomputes the stages
    ev[2].record()
    if stages:
        bwd(big)                 # stage checkpoints: the reverse sweep reads them
    ev[3].record()
    torch.cuda.synchronize()
    t_w = None
    if wide_ok:
        saved = n_acc.clone()
        ew = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ew[0].record()
        fwd(256)
        ew[1].record()
        torch.cuda.synchronize()
        t_w = ew[0].elapsed_time(ew[1]) / 1e3
        n_acc.copy_(saved)
    t_f = ev[0].elapsed_time(ev[1]) / 1e3
    t_rc = ev[1].elapsed_time(ev[2]) / 1e3
    t_b = ev[2].elapsed_time(ev[3]) / 1e3 if stages else t_rc
    out = {"workload": "adjoint_front_heavy_%d_cells_dt1e-8" % n, "cells": n, "forward_s": t_f, "adjoint_s": t_b,
           "ratio": t_b / t_f, "memory_mode": "stage checkpoints" if stages else "step checkpoints, stages recomputed",
           "adjoint_recompute_s": t_rc, "ratio_recompute": t_rc / t_f, "accepted_steps": total,
           "workspace_GB": (big if stages else small) / 1e9, "workspace_recompute_GB": small / 1e9,
           "adjoint_cell_steps_per_s": n / t_b,
           "forward_wide_s": t_w, "ratio_vs_wide_forward": (t_b / t_w) if t_w else None,
           "forward_note": "forward_s: the 128-thread kernel, whose arithmetic the adjoint retraces; "
                           "forward_wide_s: the wide 256-thread queue kernel, the fastest forward",
           "grad_norms": {"gT0": float(gT0.norm()), "glnA": float(glnA.norm()), "gE": float(gE.norm())}}
    m.close()
    del ws
    torch.cuda.empty_cache()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cells", type=int, default=FIELD_CELLS)
    ap.add_argument("--schedule", default="queue", choices=["queue", "plain"])
    ap.add_argument("--ctas-per-sm", type=int, default=0)
    ap.add_argument("--threads", type=int, default=256, choices=[0, 128, 256],
                    help="threads per CTA of the queue kernel: 256 = the wide queue kernel (default: the "
                         "faster one on the 2,097,152-cell field), 0 = library choice (128), 128")
    ap.add_argument("--no-compare-narrow", action="store_true",
                    help="skip timing the queue kernel of the other CTA width (128 or 256 threads)")
    ap.add_argument("--order", default="index", choices=["cost", "index", "hot", "pT"],
                    help="queue order: by cell index (default); by the previous step's attempts, most first "
                         "(cost; every timed step restarts from the same state, so that order knows the step's "
                         "own costs in advance); or from the step's own input: hottest cells first (hot), "
                         "highest p T first (pT)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-compare-plain", action="store_true",
                    help="skip timing the plain schedule (one thread per cell, one pass) against the queue")
    ap.add_argument("--plain-steps", type=int, default=2, help="steps of the plain-schedule comparison")
    ap.add_argument("--no-amr", action="store_true", help="skip the 64-block AMR graph leg")
    ap.add_argument("--partition", default="cost", choices=["cost", "replicas"],
                    help="N > 1: split one field across the ranks by the previous step's measured per-cell "
                         "cycles (cost; strong scaling), or give every rank its own field (replicas; weak)")
    ap.add_argument("--workload", default="field", choices=["field", "amr_graph", "large_field", "methods"])
    ap.add_argument("--amr-steps", type=int, default=100)
    ap.add_argument("--curve", action="store_true", help="amr_graph: also time each step eagerly")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--adjoint-cells", type=int, default=ADJ_CELLS)
    ap.add_argument("--no-large", action="store_true", help="skip the 53-species stress leg")
    ap.add_argument("--generic", action="store_true", help="use the precompiled kernels, not the specialised ones")
    ap.add_argument("--large-sample", type=int, default=LARGE_SAMPLE)
    args = ap.parse_args()
    world, rank, local = dist_setup()
    if args.impl == "reference":
        return reference_arm(args, world, rank)
    if args.workload == "amr_graph":
        return amr_graph_workload(args) if rank == 0 else 0
    if args.workload == "methods":
        return methods_workload(args) if rank == 0 else 0
    if args.workload == "large_field":
        if rank == 0:
            from paper_2508_16105_gb300 import build, rde_chem
            build.build_library()
            rde_chem.load_library()
            leg = large_field_leg(args.steps, args.warmup, args.large_sample)
            leg["lu54_tensor_vs_cuda_core"] = lu54_leg()
            leg["adjoint"] = large_adjoint_leg()
            out = {"metric": "cell-chemistry steps/s (FP64, 53-species stress mechanism)", "value": leg["value"],
                   "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
                   "ms_per_step": leg["kernel_ms"], "higher_is_better": True, "scaling": "weak",
                   "vs_baseline": None, "dtype": "f64", "data": "synthetic", "gpu_launches": args.steps,
                   "config": {"workload": leg["workload"], "cells": leg["cells_sampled"],
                              "species": leg["species"], "reactions": leg["reactions"], "dt": DT},
                   "roofline": leg["roofline"], "large": leg}
            print(json.dumps(out), flush=True)
        return 0

    import torch
    from paper_2508_16105_gb300 import build, rde_chem, roofline, shard, synth

    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    build.build_library()
    rde_chem.load_library()
    mech = synth.h2_air_mechanism(MECH_SEED)
    n = args.cells
    # N > 1: one field split across the ranks by the previous step's measured per-cell
    # cycles (the paper's time-weighted balancing of ranks; only those costs cross ranks),
    # or independent replica fields
    partition = "none" if world == 1 else args.partition
    field = synth.field_cells(mech, n, seed=FIELD_SEED + (rank if partition == "replicas" else 0))
    K = mech.K
    dev = torch.device("cuda", local)
    p = torch.as_tensor(field.p, device=dev)
    T0 = torch.as_tensor(field.T, device=dev)
    Y0 = torch.as_tensor(np.ascontiguousarray(field.Y), device=dev)
    T = T0.clone()
    Y = Y0.clone()
    m = rde_chem.Mechanism(mech.to_text(), flags=rde_chem.RDE_LOAD_GENERIC if args.generic else 0)
    variant, jit_s = rde_chem.rde_chem_kernel_variant(m.handle)
    specialized = variant == rde_chem.RDE_KERNEL_SPECIALIZED
    wide = specialized and args.schedule == "queue" and args.threads == 256
    if wide:
        kname = "rde_jit_queue_w (specialised to the mechanism, 256 threads per CTA)"
    else:
        kname = ("rde_jit_%s (specialised to the mechanism)" if specialized else
                 "chem_advance_kernel<9,%s>") % args.schedule
    sched = rde_chem.RDE_SCHED_QUEUE if args.schedule == "queue" else rde_chem.RDE_SCHED_PLAIN
    stream = torch.cuda.current_stream()
    # per-cell attempt counts of each step; with --order cost the next step's queue hands
    # out the cells by them, most expensive first
    n_acc = torch.zeros(n, dtype=torch.int32, device=dev)
    n_rej = torch.zeros(n, dtype=torch.int32, device=dev)
    cyc = torch.zeros(n, dtype=torch.int64, device=dev)
    ranges = [shard.even_ranges(n, world)]
    imbalances = []

    def my_range():
        return ranges[0][rank] if partition == "cost" else (0, n)

    def make_blk(pp, TT, YY):
        lo, hi = my_range()
        return rde_chem.make_block(pp[lo:], TT[lo:], YY[:, lo:], n_acc=n_acc[lo:], n_rej=n_rej[lo:],
                                   cycles=cyc[lo:], n=hi - lo, ldY=n)

    by_cost = args.order == "cost" and partition == "none"
    by_heat = args.order in ("hot", "pT") and partition == "none"
    heat_key = (-T0 if args.order == "hot" else -(p * T0)) if by_heat else None
    order = [None]
    k0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    k1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]

    def rebalance():
        if partition == "cost":
            lo, hi = my_range()
            new, loads, imb = shard.repartition(cyc[lo:hi].to(torch.float64), ranges[0], world)
            ranges[0] = new
            imbalances.append(imb)

    def step(i=None, schedule=sched, threads=None):
        T.copy_(T0)
        Y.copy_(Y0)
        if i is not None:
            k0[i].record(stream)
        thr = args.threads if threads is None else threads
        if by_heat:   # from the step's own input only
            order[0] = torch.argsort(heat_key, stable=True)
        rde_chem.rde_chem_advance_ex(m.handle, DT, cells=make_blk(p, T, Y), schedule=schedule,
                                     ctas_per_sm=args.ctas_per_sm, order=order[0], stream=stream,
                                     threads_per_cta=0 if schedule == rde_chem.RDE_SCHED_PLAIN else thr)
        if i is not None:
            k1[i].record(stream)
        if by_cost:
            order[0] = torch.argsort(-(n_acc + n_rej), stable=True)
        rebalance()

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    for _ in range(args.warmup):
        step()
    uuid = None
    try:
        uuid = str(torch.cuda.get_device_properties(dev).uuid)
        uuid = uuid if uuid.startswith("GPU-") else "GPU-" + uuid
    except Exception:
        uuid = None
    clocks = ClockSampler(uuid)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for i in range(args.steps):
        step(i)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    elapsed = e0.elapsed_time(e1) / 1e3
    kernel_s = [a.elapsed_time(b) / 1e3 for a, b in zip(k0, k1)]
    stats = rde_chem.rde_chem_get_stats(m.handle)
    if world > 1:
        t = torch.tensor([elapsed], device=dev, dtype=torch.float64)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        elapsed = float(t.item())
    # cells all ranks advanced per step: the one field (cost partition) or one per rank
    value = (n if partition == "cost" else world * n) * args.steps / elapsed

    # roofline of the chemistry kernel (algorithmic flops / measured launch time); exp, log,
    # division and root count 1 flop (the primary figure), or their FP64 cost (weighted)
    fl = roofline.flops_per_attempt(mech)
    flw = roofline.flops_per_attempt(mech, weighted=True)
    attempts = stats["accepted"] + stats["rejected"]
    k_avg = float(np.mean(kernel_s))
    achieved = fl["total"] * attempts / k_avg / 1e9
    achieved_w = flw["total"] * attempts / k_avg / 1e9
    tkey = kernel_source_hash() + ("/w" if wide else "/n")
    traffic = TRAFFIC_BYTES_PER_CELL.get(tkey) if specialized else None   # measured on the specialised kernel
    roof = {"bound": "alu", "achieved": achieved, "peak": roofline.FP64_PEAK_GFLOPS, "unit": "GFLOP/s",
            "frac": achieved / roofline.FP64_PEAK_GFLOPS,
            "traffic": traffic * n if traffic is not None else None,
            "peak_source": "FP64 2 DFMA/clk/SM x 152 SMs x 2070 MHz (recipe unit counts); DFMA microbenchmark "
                           "measured %.0f GFLOP/s" % roofline.FP64_MEASURED_GFLOPS,
            "kernel": kname, "kernel_ms": 1e3 * k_avg,
            "flops_per_attempt": fl["total"], "flop_rule": "exp, log, division and root = 1 flop; FMA = 2",
            "attempts_per_launch": attempts,
            "weighted": {"flops_per_attempt": flw["total"], "achieved": achieved_w,
                         "frac": achieved_w / roofline.FP64_PEAK_GFLOPS,
                         "flop_rule": "exp, log = 16 flops, division, root = 8 (their FP64 arithmetic)"},
            "algorithmic_bytes_per_launch": roofline.algorithmic_bytes_per_cell(K) * n}
    xf = EXECUTED_FLOPS_PER_ATTEMPT.get(tkey) if specialized else None
    roof["ncu_executed"] = None if xf is None else {
        "flops_per_attempt": xf, "achieved": xf * attempts / k_avg / 1e9,
        "frac": xf * attempts / k_avg / 1e9 / roofline.FP64_PEAK_GFLOPS,
        "rule": "2 dfma + dadd + dmul thread instructions per attempt from one ncu capture of this kernel on "
                "this field, times this run's attempts, over this run's kernel time"}

    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": 1e3 * elapsed / args.steps, "higher_is_better": True,
           "scaling": "strong" if partition == "cost" else "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic",
           "config": {"workload": "rde_field_2d_h2air_9sp21rx_dt5e-9", "cells": n, "species": K,
                      "reactions": mech.R, "dt": DT, "rtol": 1e-8, "atol": 1e-12, "schedule": args.schedule,
                      "threads_per_cta": 256 if wide else 128,
                      "mix": "90% fresh / 5% front / 5% burnt", "seed": FIELD_SEED,
                      "queue_order": ("cells by the previous step's attempts, most first (the argsort is inside "
                                      "the timed step)" if by_cost else
                                      ("hottest cells first" if args.order == "hot" else "highest p T first") +
                                      " (argsort of the step's input inside the timed step)" if by_heat else
                                      "cell index"),
                      "kernel_variant": "specialised" if specialized else "generic",
                      "parallelism": ("one field split by measured per-cell cycles (time-weighted ranges, "
                                      "re-cut after every step)" if partition == "cost" else
                                      "replica fields, one per rank" if partition == "replicas" else "1 GPU"),
                      "l2": "inputs larger than L2 (%d MB of p, T, Y re-copied every step)" % (n * (K + 2) * 8 // 2**20)},
           "roofline": roof, "gpu_launches": args.steps,
           "substeps_per_cell": attempts / n, "failed_cells": stats["failed"],
           "adjoint_forward_ratio": None, "clocks": clk, "load_compile_s": jit_s}

    if not args.no_compare_plain and rank == 0:
        # the same steps with the plain schedule (one thread per cell, one pass, no queue)
        ns = max(1, min(args.steps, args.plain_steps))
        saved = order[0]
        order[0] = None
        for i in range(ns):
            step(i, schedule=rde_chem.RDE_SCHED_PLAIN)
        torch.cuda.synchronize()
        order[0] = saved
        plain_ms = float(np.mean([k0[i].elapsed_time(k1[i]) for i in range(ns)]))
        out["schedules"] = {"queue_schedule_ms": 1e3 * k_avg, "plain_schedule_ms": plain_ms,
                            "plain_over_queue": plain_ms / (1e3 * k_avg), "plain_steps": ns,
                            "queue_steps": args.steps,
                            "plain": "one thread per cell, grid of ceil(n/128) CTAs, one pass",
                            "queue": "persistent CTAs, lanes refilled from a device work queue"}
    if specialized and args.schedule == "queue" and not args.no_compare_narrow and rank == 0:
        # the same steps with the other CTA width: the wide 256-thread queue kernel beside the
        # 128-thread one (every lane slot in shared memory), or the reverse with --threads 256
        ns = max(1, min(args.steps, args.plain_steps))
        step(None, threads=128 if wide else 256)   # first use of the other width (the wide one compiles)
        torch.cuda.synchronize()
        for i in range(ns):
            step(i, threads=128 if wide else 256)
        torch.cuda.synchronize()
        other_ms = float(np.mean([k0[i].elapsed_time(k1[i]) for i in range(ns)]))
        wide_ms, narrow_ms = (1e3 * k_avg, other_ms) if wide else (other_ms, 1e3 * k_avg)
        out["cta_width"] = {"wide_ms": wide_ms, "narrow_ms": narrow_ms, "narrow_over_wide": narrow_ms / wide_ms,
                            "steps": ns,
                            "wide": "rde_jit_queue_w: 256 threads per CTA, matrix in shared memory, species and "
                                    "vector slots in registers (two warps per SM sub-partition)",
                            "narrow": "rde_jit_queue: 128 threads per CTA, every lane slot in shared memory"}
    if not args.no_e2e:
        # end to end through the C ABI from pinned host buffers: H2D inputs, advance, D2H results
        # (with a cost partition, each rank copies its current range of cells in and out)
        hp = torch.as_tensor(field.p).pin_memory()
        hT = torch.as_tensor(field.T).pin_memory()
        hY = torch.as_tensor(np.ascontiguousarray(field.Y)).pin_memory()
        oT = torch.empty_like(hT).pin_memory()
        oY = torch.empty_like(hY).pin_memory()
        dp, dT, dY = torch.empty_like(p), torch.empty_like(T), torch.empty_like(Y)
        moved = [0, 0]

        def e2e_step():
            lo, hi = my_range()
            dp[lo:hi].copy_(hp[lo:hi], non_blocking=True)
            dT[lo:hi].copy_(hT[lo:hi], non_blocking=True)
            dY[:, lo:hi].copy_(hY[:, lo:hi], non_blocking=True)
            rde_chem.rde_chem_advance_ex(m.handle, DT, cells=make_blk(dp, dT, dY), schedule=sched, order=order[0],
                                         stream=stream, threads_per_cta=args.threads)
            oT[lo:hi].copy_(dT[lo:hi], non_blocking=True)
            oY[:, lo:hi].copy_(dY[:, lo:hi], non_blocking=True)
            moved[0] = 8 * (hi - lo) * (K + 2)
            moved[1] = 8 * (hi - lo) * (K + 1)
            if by_cost:
                order[0] = torch.argsort(-(n_acc + n_rej), stable=True)
            rebalance()

        e2e_step()
        torch.cuda.synchronize()
        barrier()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        ns = max(1, min(args.steps, 3))
        for _ in range(ns):
            e2e_step()
        b.record(stream)
        torch.cuda.synchronize()
        te = a.elapsed_time(b) / 1e3
        if world > 1:
            t = torch.tensor([te], device=dev, dtype=torch.float64)
            torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
            te = float(t.item())
        out["e2e"] = {"value": (n if partition == "cost" else world * n) * ns / te, "unit": UNIT, "steps": ns,
                      "h2d_bytes_per_step": moved[0], "d2h_bytes_per_step": moved[1]}
        out["gpu_launches_e2e"] = ns

    if partition == "cost":
        out["partition"] = {"final_ranges": ranges[0], "imbalance_per_step": [round(x, 4) for x in imbalances],
                            "cost": "per-cell SM clock cycles of the previous step (rde_block.cycles)"}
    if rank == 0 and not args.no_adjoint:
        adj = adjoint_leg(mech, args.adjoint_cells)
        out["adjoint_forward_ratio"] = adj["ratio"]
        out["adjoint"] = adj
    if rank == 0 and not args.no_amr:
        out["amr_graph"] = amr_graph_leg(args.amr_steps, 1, True, threads=args.threads)
    if rank == 0 and not args.no_large:
        out["stress_53sp"] = large_field_leg(1, 1, args.large_sample)
        out["stress_53sp"]["lu54_tensor_vs_cuda_core"] = lu54_leg()
        out["stress_53sp"]["adjoint"] = large_adjoint_leg()
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(mech, field, min(CPU_SAMPLE, n))
    m.close()
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
