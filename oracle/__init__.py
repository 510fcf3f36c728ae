"""CPU oracle for the per-cell chemistry step (serial, FP64).

TEST INFRASTRUCTURE ONLY.  Only tests/, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The product path (the CUDA library and its Python binding) never
imports it; the two share no code.

The C source (oracle.c) is compiled with gcc into ``oracle/_build`` by
``build_oracle()`` with ``-ffp-contract=off`` so that every operation rounds
as written on both x86-64 and aarch64 hosts.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor

import numpy as np

from .mech import OracleMech, RU  # noqa: F401

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_SRCS = [os.path.join(_HERE, n) for n in ("oracle.c", "oracle_cs.c", "oracle.h")]
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

STATUS = {0: "OK", 1: "MAX_SUBSTEPS", 2: "H_UNDERFLOW", 3: "BAD_STATE", 4: "LU_SINGULAR"}


def build_oracle(force: bool = False) -> str:
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(os.path.getmtime(f) for f in _SRCS):
        tmp = _LIB + ".%d.tmp" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                               "-o", tmp, _SRCS[0], _SRCS[1], "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Mech(C.Structure):
    _fields_ = [("K", C.c_int), ("R", C.c_int),
                ("W", C.c_void_p), ("Tmid", C.c_void_p), ("lo", C.c_void_p), ("hi", C.c_void_p),
                ("type", C.c_void_p), ("rev", C.c_void_p), ("nuf", C.c_void_p), ("nur", C.c_void_p),
                ("A", C.c_void_p), ("b", C.c_void_p), ("EaR", C.c_void_p),
                ("A0", C.c_void_p), ("b0", C.c_void_p), ("EaR0", C.c_void_p),
                ("troe", C.c_void_p), ("ntroe", C.c_void_p), ("eff", C.c_void_p)]


class Opts(C.Structure):
    _fields_ = [("rtol", C.c_double), ("atol", C.c_double), ("hmin", C.c_double),
                ("facmax", C.c_double), ("facmin", C.c_double), ("safety", C.c_double),
                ("max_substeps", C.c_int), ("method", C.c_int)]


METHOD_RODAS3, METHOD_ROS2, METHOD_EXTRAP = 0, 1, 2


def default_opts(rtol=1e-8, atol=1e-12, max_substeps=100000, method=METHOD_RODAS3) -> Opts:
    return Opts(rtol, atol, 1e-30, 5.0, 0.2, 0.9, max_substeps, method)


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build_oracle())
            P = C.c_void_p
            lib.orc_rhs.argtypes = [P, C.c_double, P, P]
            lib.orc_jac.argtypes = [P, C.c_double, P, P, P]
            lib.orc_rates.argtypes = [P, C.c_double, P, P, P, P]
            lib.orc_thermo.argtypes = [P, C.c_int, C.c_double, P, P, P]
            lib.orc_tableau.argtypes = [P, P, P, P, P]
            lib.orc_lu_solve.argtypes = [C.c_int, P, P, P, C.c_int]
            lib.orc_fixed_step.argtypes = [P, C.c_double, P, C.c_double, P, P]
            lib.orc_fixed_step_method.argtypes = [P, C.c_int, C.c_double, P, C.c_double, P, P]
            lib.orc_tableau_method.argtypes = [C.c_int, P, P, P, P, P, P]
            lib.orc_advance.argtypes = [P, P, C.c_long, P, P, P, C.c_long, C.c_double, P, P, P, P]
            lib.orc_advance_record.argtypes = [P, P, C.c_double, P, C.c_double, P, C.c_int, P]
            lib.orc_replay.argtypes = [P, C.c_double, P, P, C.c_int]
            lib.orc_tangent.argtypes = [P, C.c_double, P, P, P, P, P, C.c_int, P, P]
            _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data


class Oracle:
    """Serial FP64 reference integrator for one mechanism."""

    def __init__(self, mech_text: str):
        self.lib = _load()
        self.m = OracleMech(mech_text)
        m = self.m
        self._keep = [np.ascontiguousarray(x) for x in
                      (m.W, m.Tmid, m.lo, m.hi, m.type, m.rev, m.nuf, m.nur, m.A, m.b, m.EaR,
                       m.A0, m.b0, m.EaR0, m.troe, m.ntroe, m.eff)]
        self.cm = _Mech(m.K, m.R, *[_ptr(a) for a in self._keep])
        self.K, self.R, self.N = m.K, m.R, m.K + 1

    @property
    def _mp(self):
        return C.addressof(self.cm)

    def rhs(self, p: float, y: np.ndarray) -> np.ndarray:
        y = np.ascontiguousarray(y, dtype=np.float64)
        f = np.empty(self.N)
        self.lib.orc_rhs(self._mp, p, _ptr(y), _ptr(f))
        return f

    def jac(self, p: float, y: np.ndarray):
        y = np.ascontiguousarray(y, dtype=np.float64)
        f = np.empty(self.N)
        J = np.empty((self.N, self.N))
        self.lib.orc_jac(self._mp, p, _ptr(y), _ptr(f), _ptr(J))
        return f, J

    def rates(self, p: float, y: np.ndarray):
        y = np.ascontiguousarray(y, dtype=np.float64)
        kf, kr, q = np.empty(self.R), np.empty(self.R), np.empty(self.R)
        self.lib.orc_rates(self._mp, p, _ptr(y), _ptr(kf), _ptr(kr), _ptr(q))
        return kf, kr, q

    def thermo(self, k: int, T: float):
        v = (C.c_double(), C.c_double(), C.c_double())
        self.lib.orc_thermo(self._mp, k, T, *[C.byref(x) for x in v])
        return tuple(x.value for x in v)

    def fixed_step(self, p: float, y: np.ndarray, h: float, method: int = METHOD_RODAS3):
        y = np.ascontiguousarray(y, dtype=np.float64)
        yn, e = np.empty(self.N), np.empty(self.N)
        rc = self.lib.orc_fixed_step_method(self._mp, method, p, _ptr(y), h, _ptr(yn), _ptr(e))
        return rc, yn, e

    def advance(self, p, T, Y, dt, opts: Opts | None = None, hint=None, threads: int = 1):
        """Advance cells in place-free fashion; returns (T, Y, status, nacc, nrej, hint)."""
        opts = opts or default_opts()
        p = np.ascontiguousarray(p, dtype=np.float64)
        T = np.array(T, dtype=np.float64, copy=True)
        Y = np.array(Y, dtype=np.float64, copy=True, order="C")
        n = T.shape[0]
        hint = None if hint is None else np.array(hint, dtype=np.float64, copy=True)
        st = np.zeros(n, np.int32)
        na = np.zeros(n, np.int32)
        nr = np.zeros(n, np.int32)
        ldY = Y.shape[1] if Y.ndim == 2 else n

        def run(lo, hi):
            if hi <= lo:
                return
            off = lambda a, esz=8: None if a is None else a.ctypes.data + lo * esz
            self.lib.orc_advance(self._mp, C.addressof(opts), hi - lo, off(p), off(T), off(Y), ldY, dt,
                                 off(hint), off(st, 4), off(na, 4), off(nr, 4))

        if threads <= 1 or n < 2 * threads:
            run(0, n)
        else:
            chunk = max(1, (n + 4 * threads - 1) // (4 * threads))
            with ThreadPoolExecutor(threads) as ex:
                list(ex.map(lambda lo: run(lo, min(n, lo + chunk)), range(0, n, chunk)))
        return T, Y, st, na, nr, hint


class FrozenSteps:
    """Accepted step sizes of one cell's adaptive integration (the frozen sequence)."""

    def __init__(self, h):
        self.h = np.ascontiguousarray(h, dtype=np.float64)

    def __len__(self):
        return len(self.h)


def record(o: "Oracle", p: float, y0, dt: float, opts: Opts | None = None, cap: int = 200000):
    """Adaptive integration of one cell recording its accepted steps -> (status, y_end, FrozenSteps)."""
    opts = opts or default_opts()
    y = np.array(y0, dtype=np.float64, copy=True)
    h = np.empty(cap)
    n = C.c_int()
    rc = o.lib.orc_advance_record(o._mp, C.addressof(opts), p, _ptr(y), dt, _ptr(h), cap, C.byref(n))
    return rc, y, FrozenSteps(h[:n.value])


def replay(o: "Oracle", p: float, y0, steps: FrozenSteps, dlnA=None, dE=None):
    """Frozen-step map in real arithmetic; dlnA / dE (per reaction) perturb ln A_r and E_r (J/mol)."""
    y = np.array(y0, dtype=np.float64, copy=True)
    if dlnA is not None or dE is not None:
        # perturb the oracle's SI pre-factors / activation temperatures, replay, restore
        A0, E0 = o.m.A.copy(), o.m.EaR.copy()
        kA, kE = o._keep[8], o._keep[10]
        if dlnA is not None:
            kA[:] = A0 * np.exp(np.asarray(dlnA))
        if dE is not None:
            kE[:] = E0 + np.asarray(dE) / RU
        rc = o.lib.orc_replay(o._mp, p, _ptr(y), _ptr(steps.h), len(steps))
        kA[:] = A0
        kE[:] = E0
    else:
        rc = o.lib.orc_replay(o._mp, p, _ptr(y), _ptr(steps.h), len(steps))
    return rc, y


def tangent(o: "Oracle", p: float, y0, steps: FrozenSteps, dy0=None, dlnA=None, dE=None):
    """Exact directional derivative of the frozen-step map (complex step) -> (y_end, dy_end)."""
    y0 = np.ascontiguousarray(y0, dtype=np.float64)
    yo, dyo = np.empty(o.N), np.empty(o.N)
    arr = lambda a: None if a is None else np.ascontiguousarray(a, dtype=np.float64)
    dy0, dlnA, dE = arr(dy0), arr(dlnA), arr(dE)
    rc = o.lib.orc_tangent(o._mp, p, _ptr(y0), _ptr(dy0), _ptr(dlnA), _ptr(dE), _ptr(steps.h), len(steps),
                           _ptr(yo), _ptr(dyo))
    assert rc == 0
    return yo, dyo


def tableau():
    lib = _load()
    g = C.c_double()
    a, c, m, e = np.empty(16), np.empty(16), np.empty(4), np.empty(4)
    lib.orc_tableau(C.byref(g), _ptr(a), _ptr(c), _ptr(m), _ptr(e))
    return g.value, a.reshape(4, 4), c.reshape(4, 4), m, e


def tableau_method(method: int):
    """(stages, gamma, a, c, m, e, qhat) of a method (0: RODAS3, 1: ROS2), transformed form."""
    lib = _load()
    g, q = C.c_double(), C.c_int()
    a, c, m, e = np.empty(16), np.empty(16), np.empty(4), np.empty(4)
    s = lib.orc_tableau_method(method, C.byref(g), _ptr(a), _ptr(c), _ptr(m), _ptr(e), C.byref(q))
    return s, g.value, a.reshape(4, 4)[:s, :s], c.reshape(4, 4)[:s, :s], m[:s], e[:s], q.value


def lu_solve(A: np.ndarray, B: np.ndarray):
    lib = _load()
    N = A.shape[0]
    a = np.array(A, dtype=np.float64, copy=True, order="C")
    x = np.array(B, dtype=np.float64, copy=True, order="C").reshape(-1, N)
    piv = np.zeros(N, np.int32)
    rc = lib.orc_lu_solve(N, _ptr(a), _ptr(piv), _ptr(x), x.shape[0])
    return rc, x
