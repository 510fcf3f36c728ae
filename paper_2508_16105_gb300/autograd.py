"""torch.autograd.Function over the chemistry step.

Forward advances the cells with the sm_103a kernel (recording each cell's
accepted step count); backward calls the library's discrete adjoint, which
re-integrates every cell, records its accepted steps and sweeps them backwards.
Gradients flow to T0, Y0 and to the mechanism's Arrhenius parameters ln A_r and
E_r (J/mol), which enter as tensors: their values are written into the
mechanism tables before the step, so the function can be used for calibration.
The forward keeps a host copy of the parameters it ran with; backward puts them
back into the tables for the adjoint and afterwards restores whatever the tables
held, so several steps on one mechanism (time steps, or parameter sets) each
differentiate at their own parameters.
With stages=True the backward allocates the larger workspace that holds every
accepted step's LU factors and stage vectors (stage checkpoints), and the
reverse sweep reads them instead of recomputing them.
Only argument marshalling happens here; every step runs in the library.
"""
from __future__ import annotations

import torch

from . import rde_chem


class ChemStep(torch.autograd.Function):
    @staticmethod
    def forward(ctx, mech: "rde_chem.Mechanism", dt: float, p, T0, Y0, lnA, E, stages: bool = False):
        lnA_h = lnA.detach().double().cpu().numpy().copy()
        E_h = E.detach().double().cpu().numpy().copy()
        rde_chem.rde_mech_set_arrhenius(mech.handle, lnA_h, E_h)
        T = T0.detach().clone()
        Y = Y0.detach().clone().contiguous()
        n = int(T.shape[0])
        n_acc = torch.zeros(n, dtype=torch.int32, device=T.device)
        status = torch.zeros(n, dtype=torch.int32, device=T.device)
        # the 128-thread kernels: the arithmetic the adjoint's re-integration retraces, so the
        # recorded step counts match it
        rde_chem.rde_chem_advance_ex(mech.handle, dt, cells=rde_chem.make_block(p, T, Y, n_acc=n_acc, status=status),
                                     threads_per_cta=128)
        ctx.save_for_backward(p, T0.detach(), Y0.detach().contiguous(), n_acc)
        ctx.mech = mech
        ctx.params = (lnA_h, E_h)
        ctx.dt = dt
        ctx.stages = bool(stages)
        ctx.mark_non_differentiable(status)
        return T, Y, status

    @staticmethod
    def backward(ctx, gT, gY, _gstatus):
        p, T0, Y0, n_acc = ctx.saved_tensors
        mech = ctx.mech
        gT = torch.zeros_like(T0) if gT is None else gT.contiguous()
        gY = torch.zeros_like(Y0) if gY is None else gY.contiguous()
        n = int(T0.shape[0])
        total = int(n_acc.sum().item())
        size = (rde_chem.rde_chem_adjoint_workspace_checkpointed if ctx.stages else
                rde_chem.rde_chem_adjoint_workspace_steps)(mech.handle, n, total)
        ws = torch.empty(size, dtype=torch.uint8, device=T0.device)
        gT0 = torch.empty_like(T0)
        gY0 = torch.empty_like(Y0)
        glnA = torch.empty(mech.R, dtype=torch.float64, device=T0.device)
        gE = torch.empty(mech.R, dtype=torch.float64, device=T0.device)
        current = rde_chem.rde_mech_get_arrhenius(mech.handle, mech.R)
        rde_chem.rde_mech_set_arrhenius(mech.handle, *ctx.params)
        try:
            rde_chem.rde_chem_advance_adjoint_ex(mech.handle, ctx.dt, p, T0, Y0, n_acc, total, gT, gY, gT0, gY0, glnA,
                                              gE, ws)
        finally:
            rde_chem.rde_mech_set_arrhenius(mech.handle, *current)   # waits for the adjoint's kernels
        return None, None, None, gT0, gY0, glnA, gE, None


def chem_step(mech, dt, p, T0, Y0, lnA, E, stages: bool = False):
    """Differentiable step: returns (T, Y, status); stages selects stage checkpoints."""
    return ChemStep.apply(mech, dt, p, T0, Y0, lnA, E, stages)
