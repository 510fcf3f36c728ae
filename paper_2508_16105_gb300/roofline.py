"""Algorithmic FP64 work of one Rosenbrock attempt, for roofline accounting.

The count follows the operations the method needs (not what a kernel happens
to issue): additions and multiplications count 1 flop, a fused multiply-add 2,
and an exponential, logarithm, division, reciprocal, square or cube root 1
(the primary count, ``flops_per_attempt(mech)``).  A secondary count weighs
what such an operation costs in FP64 arithmetic on this GPU:
``flops_per_attempt(mech, weighted=True)`` charges a division or root 8 flops (a
Newton-refined reciprocal) and an exponential or logarithm 16 (the table-driven
evaluation: argument reduction plus a degree-4 polynomial, seven fused
multiply-adds and two further operations).  One attempt of
RODAS3 is: f and the analytic Jacobian at y_n, the matrix I/(h gamma) - J, its
LU factorisation with partial pivoting, four triangular solves, two further f
evaluations (stages 3 and 4; stage 2 reuses f(y_n)), the stage combinations and
the error norm with the step-size update.

Peak: GB300 retires two FP64 fused multiply-adds per SM per clock (4 flops),
152 SMs at 2070 MHz: 1258.6 GFLOP/s.  A DFMA-only microbenchmark reached
1200 GFLOP/s (95.4 %) at 2070 MHz on this GPU.
"""
from __future__ import annotations

WEIGHTED_TRANS = 16   # flops charged for exp / log in the weighted count
WEIGHTED_DIV = 8      # flops charged for a division or root in the weighted count

FP64_PEAK_GFLOPS = 2 * 2 * 152 * 2.070     # 1258.56: 2 DFMA/clk/SM x 2 flop x 152 SMs x 2.07 GHz
FP64_MEASURED_GFLOPS = 1200.0              # DFMA microbenchmark on GB300


def _reaction_terms(r):
    nf, nb = len(r.reac), len(r.prod)
    of = sum(c for _, c in r.reac)
    ob = sum(c for _, c in r.prod)
    net = {}
    for n, c in r.reac:
        net[n] = net.get(n, 0) - c
    for n, c in r.prod:
        net[n] = net.get(n, 0) + c
    npart = sum(1 for v in net.values() if v != 0)
    neff = sum(1 for a in r.eff.values() if a != 1.0) if r.kind != "ELEM" else 0
    return nf, nb, of, ob, npart, neff


def flops_per_attempt(mech, weighted: bool = False) -> dict:
    """Algorithmic flops of one attempt for a ``synth.Mechanism`` (K species, R reactions).

    Exponentials, logarithms, divisions and roots count 1 flop each, or, with
    ``weighted``, 16 (exp, log) and 8 (division, root)."""
    FLOP_TRANS = WEIGHTED_TRANS if weighted else 1
    FLOP_DIV = WEIGHTED_DIV if weighted else 1
    K = mech.K
    N = K + 1
    # ---- one f evaluation ----
    f_mix = 4 * K + 3 + FLOP_DIV
    f_thermo = 32 * K + FLOP_TRANS + FLOP_DIV
    f_rx = 0
    j_rx = 0
    for r in mech.reactions:
        nf, nb, of, ob, npart, neff = _reaction_terms(r)
        c = 4 + FLOP_TRANS                           # ln k and k
        c += 2 * neff                                # [M] corrections
        if r.kind in ("LINDEMANN", "TROE"):
            c += 4 + FLOP_TRANS + 2 + FLOP_DIV + 10  # k0, Pr, Lindemann blend
            if r.kind == "TROE":
                c += 3 * FLOP_TRANS + 2 * FLOP_TRANS + 10 + FLOP_DIV + FLOP_TRANS
        if r.reversible:
            c += 2 * (nf + nb) + 2 + FLOP_TRANS + 1
        c += (of - 1) + (ob - 1) + 3 + (1 if r.kind == "THREEBODY" else 0)
        c += 2 * npart
        f_rx += c
        # Jacobian-only work of this reaction
        jc = 3 + 6 + 2 * npart                       # d ln kf/dT, dq/dT, wT
        if r.reversible:
            jc += 2 * (nf + nb) + 2
        jc += 3 * (nf + nb)                          # d(product)/dc
        jc += 2 * npart * (nf + nb)                  # D updates
        if r.kind != "ELEM":
            jc += npart * (K + 2 * neff) + 2
        if r.kind in ("LINDEMANN", "TROE"):
            jc += 12 + (30 if r.kind == "TROE" else 0)
        j_rx += jc
    f_out = 4 * K + 3 + FLOP_DIV
    C_f = f_mix + f_thermo + f_rx + f_out
    C_J = 8 * K + j_rx + 4 * K * K + 8 * K + 3 * K * K + 11 * K + 8 * K + 12 + 2 * FLOP_DIV + N
    C_lu = sum(FLOP_DIV + (N - k - 1) + 2 * (N - k - 1) ** 2 for k in range(N))
    C_solve = 4 * (2 * N * (N - 1) + N)
    C_stage = 16 * N + FLOP_DIV
    C_err = N * (2 + FLOP_DIV + 2) + FLOP_DIV + FLOP_TRANS + FLOP_DIV + 6
    total = 3 * C_f + C_J + C_lu + C_solve + C_stage + C_err
    return dict(total=total, rhs=C_f, jac_extra=C_J, lu=C_lu, solves=C_solve, stages=C_stage, err=C_err)


def algorithmic_bytes_per_cell(K: int) -> int:
    """HBM bytes one cell-step must move: read p, T, Y_k; write T, Y_k (FP64)."""
    return 8 * ((K + 2) + (K + 1))
