"""Operator-split coupling of the chemistry step to a toy 1D reacting flow.

The paper's solver splits the stiff chemistry from transport inside each flow
time step: the species and energy equations (Eqs. 20-21 of its appendix) get
their source terms from the detailed chemistry, which advances every cell over
the flow step (Section 2.1), and it validates the solver on a 1D detonation tube
(Section 3).  This module is the smallest coupling of that kind: a first-order
finite-volume solver of the 1D multicomponent Euler equations

    d/dt [rho, rho u, rho E, rho Y_k] + d/dx [rho u, rho u^2 + p, u (rho E + p), rho u Y_k] = 0

(Rusanov fluxes, reflecting walls at both ends, ideal-gas mixture with the
mechanism's NASA-7 thermo), alternated with a chemistry operator per step
(Lie splitting):

  1. transport over dt;
  2. every cell's (T, Y) advanced over dt at its pressure by ``chem`` (the
     constant-pressure adiabatic reactor of the chemistry step), with each cell's
     step-size hint carried from the previous step;
  3. the conservative state rebuilt with rho and momentum unchanged,
     rho Y_k = rho Y_k' and rho E = rho (e(T', Y') + u^2/2).

``chem(p, T, Y, dt, hint) -> (T', Y', hint')`` is supplied by the caller: the
sm_103a library through ``library_chemistry`` (device copies per step), or any
other integrator of the same reactor.  The transport runs on the host in float64
numpy; it is a harness for the chemistry step, not part of it.
"""
from __future__ import annotations

import numpy as np

RU = 8.31446261815324      # J/(mol K)


class MixtureThermo:
    """NASA-7 mixture properties in mass units for a ``synth.Mechanism``."""

    def __init__(self, mech):
        self.K = len(mech.species)
        self.W = np.array([s.W for s in mech.species]) * 1e-3           # kg/mol
        self.lo = np.array([s.lo for s in mech.species], dtype=np.float64)
        self.hi = np.array([s.hi for s in mech.species], dtype=np.float64)
        self.Tmid = np.array([s.Tmid for s in mech.species], dtype=np.float64)

    def _coef(self, T):
        # [K, n, 7]: the range of each species at each temperature (high range at T >= Tmid)
        use_hi = T[None, :] >= self.Tmid[:, None]
        return np.where(use_hi[:, :, None], self.hi[:, None, :], self.lo[:, None, :])

    def h_cp(self, T):
        """Species specific enthalpy and heat capacity, J/kg and J/(kg K): [K, n] each."""
        a = self._coef(T)
        t = T[None, :]
        cp_R = a[..., 0] + t * (a[..., 1] + t * (a[..., 2] + t * (a[..., 3] + t * a[..., 4])))
        h_RT = (a[..., 0] + t * (a[..., 1] / 2 + t * (a[..., 2] / 3 + t * (a[..., 3] / 4 + t * a[..., 4] / 5)))
                + a[..., 5] / t)
        return RU * t * h_RT / self.W[:, None], RU * cp_R / self.W[:, None]

    def e_cv(self, T, Y):
        """Mixture internal energy (J/kg) and cv (J/(kg K))."""
        h, cp = self.h_cp(T)
        rmix = RU * (Y / self.W[:, None]).sum(axis=0)
        return (Y * h).sum(axis=0) - rmix * T, (Y * cp).sum(axis=0) - rmix

    def temperature(self, e, Y, T0, iters: int = 30):
        """T with e(T, Y) = e by Newton's method from T0."""
        T = T0.copy()
        for _ in range(iters):
            ee, cv = self.e_cv(T, Y)
            dT = (ee - e) / cv
            T = T - dT
            if np.max(np.abs(dT) / T) < 1e-14:
                break
        return T

    def pressure(self, rho, T, Y):
        return rho * RU * T * (Y / self.W[:, None]).sum(axis=0)

    def sound_speed(self, rho, T, Y):
        _, cp = self.h_cp(T)
        rmix = RU * (Y / self.W[:, None]).sum(axis=0)
        cpm = (Y * cp).sum(axis=0)
        gamma = cpm / (cpm - rmix)
        return np.sqrt(gamma * self.pressure(rho, T, Y) / rho)


class Tube:
    """A closed 1D tube of n cells (length L, m) in conservative variables."""

    def __init__(self, mech, p, T, Y, length: float, u=None):
        self.th = MixtureThermo(mech)
        self.n = len(T)
        self.dx = length / self.n
        Y = np.array(Y, dtype=np.float64)
        T = np.array(T, dtype=np.float64)
        p = np.array(p, dtype=np.float64)
        rho = p / (RU * T * (Y / self.th.W[:, None]).sum(axis=0))
        u = np.zeros(self.n) if u is None else np.asarray(u, dtype=np.float64)
        e, _ = self.th.e_cv(T, Y)
        self.rho = rho
        self.mom = rho * u
        self.E = rho * (e + 0.5 * u * u)
        self.rhoY = rho[None, :] * Y
        self.T = T.copy()           # last temperature (Newton start and output)
        self.hint = np.zeros(self.n)

    # ---- primitive variables ----
    def primitives(self):
        rho = self.rho
        u = self.mom / rho
        Y = self.rhoY / rho[None, :]
        e = self.E / rho - 0.5 * u * u
        T = self.th.temperature(e, Y, self.T)
        p = self.th.pressure(rho, T, Y)
        return rho, u, T, p, Y

    def max_wave_speed(self) -> float:
        rho, u, T, p, Y = self.primitives()
        return float(np.max(np.abs(u) + self.th.sound_speed(rho, T, Y)))

    # ---- transport ----
    def transport(self, dt: float):
        rho, u, T, p, Y = self.primitives()
        c = self.th.sound_speed(rho, T, Y)
        # reflecting walls: ghost cells mirror the first and last cell with u -> -u
        def ext(a, sign=1.0):
            return np.concatenate([[sign * a[0]], a, [sign * a[-1]]])
        R, M, E = ext(self.rho), ext(self.mom, -1.0), ext(self.E)
        RY = np.concatenate([self.rhoY[:, :1], self.rhoY, self.rhoY[:, -1:]], axis=1)
        U, P, C = ext(u, -1.0), ext(p), ext(c)
        # fluxes at the n + 1 faces
        fR = R * U
        fM = M * U + P
        fE = U * (E + P)
        fY = RY * U[None, :]
        s = np.maximum(np.abs(U[:-1]) + C[:-1], np.abs(U[1:]) + C[1:])
        def face(f, q):
            return 0.5 * (f[..., :-1] + f[..., 1:]) - 0.5 * s * (q[..., 1:] - q[..., :-1])
        FR, FM, FE, FY = face(fR, R), face(fM, M), face(fE, E), face(fY, RY)
        k = dt / self.dx
        self.rho = self.rho - k * (FR[1:] - FR[:-1])
        self.mom = self.mom - k * (FM[1:] - FM[:-1])
        self.E = self.E - k * (FE[1:] - FE[:-1])
        self.rhoY = self.rhoY - k * (FY[:, 1:] - FY[:, :-1])
        self.T = T

    # ---- chemistry ----
    def react(self, chem, dt: float):
        rho, u, T, p, Y = self.primitives()
        T2, Y2, hint = chem(p, T, Y, dt, self.hint)
        e2, _ = self.th.e_cv(T2, Y2)
        self.rhoY = rho[None, :] * Y2
        self.E = rho * (e2 + 0.5 * u * u)
        self.T = np.asarray(T2, dtype=np.float64).copy()
        self.hint = np.asarray(hint, dtype=np.float64).copy()

    def step(self, dt: float, chem=None):
        """One split step: transport, then (if given) chemistry, over dt."""
        self.transport(dt)
        if chem is not None:
            self.react(chem, dt)


def library_chemistry(mech_handle, device="cuda"):
    """The chemistry operator through the sm_103a library: copies (p, T, Y, hint) to the
    device, advances every cell over dt with rde_chem_advance_ex (h_hint in and out),
    and copies T, Y and the hints back."""
    import torch

    from . import rde_chem

    def chem(p, T, Y, dt, hint):
        dp = torch.as_tensor(np.ascontiguousarray(p), device=device)
        dT = torch.as_tensor(np.ascontiguousarray(T), device=device)
        dY = torch.as_tensor(np.ascontiguousarray(Y), device=device)
        dh = torch.as_tensor(np.ascontiguousarray(hint), device=device)
        st = torch.zeros(dT.shape[0], dtype=torch.int32, device=device)
        blk = rde_chem.make_block(dp, dT, dY, h_hint=dh, status=st)
        rde_chem.rde_chem_advance_ex(mech_handle, dt, cells=blk)
        torch.cuda.synchronize()
        if int((st != 0).sum().item()):
            raise RuntimeError("chemistry step failed in %d cells" % int((st != 0).sum().item()))
        return dT.cpu().numpy(), dY.cpu().numpy(), dh.cpu().numpy()

    return chem
