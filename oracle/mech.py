"""The oracle's own reader for the ``RDEMECH 1`` mechanism text format.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  Independent of the CUDA
library's parser: it produces dense [R][K] stoichiometry tables in SI units for
the serial C oracle.

Unit conversions (mechanism files use mol-cm-s and kJ/mol):
  A_SI = A_cgs * (1e-6)^(m - 1), m = reaction order: the sum of reactant
         coefficients, plus one for a plain third-body reaction; for falloff
         reactions k_inf has order sum(nu') and k_0 order sum(nu') + 1.
  E / R_u in kelvin from E in kJ/mol; W from g/mol to kg/mol.
"""
from __future__ import annotations

import numpy as np

RU = 8.31446261815324
TYPES = {"ELEM": 0, "THREEBODY": 1, "LINDEMANN": 2, "TROE": 3}


class OracleMech:
    """Dense arrays describing one mechanism (SI units)."""

    def __init__(self, text: str):
        toks = [ln.split() for ln in text.splitlines()]
        toks = [t for t in toks if t and not t[0].startswith("#")]
        if toks[0] != ["RDEMECH", "1"]:
            raise ValueError("not an RDEMECH 1 file")
        pos = 1
        assert toks[pos][0] == "ELEMENTS"
        self.elements = toks[pos][2:2 + int(toks[pos][1])]
        pos += 1
        assert toks[pos][0] == "SPECIES"
        K = int(toks[pos][1])
        pos += 1
        self.names, W, Tmid, lo, hi, comp = [], [], [], [], [], []
        for _ in range(K):
            t = toks[pos]
            assert t[0] == "SP"
            self.names.append(t[1])
            W.append(float(t[2]) / 1000.0)
            Tmid.append(float(t[4]))
            comp.append([int(x) for x in t[6:6 + len(self.elements)]])
            assert toks[pos + 1][0] == "LO" and toks[pos + 2][0] == "HI"
            lo.append([float(x) for x in toks[pos + 1][1:8]])
            hi.append([float(x) for x in toks[pos + 2][1:8]])
            pos += 3
        idx = {n: i for i, n in enumerate(self.names)}
        assert toks[pos][0] == "REACTIONS"
        R = int(toks[pos][1])
        pos += 1
        self.K, self.R = K, R
        self.W = np.array(W)
        self.Tmid = np.array(Tmid)
        self.lo = np.array(lo)
        self.hi = np.array(hi)
        self.comp = np.array(comp, dtype=np.int32).reshape(K, len(self.elements))
        self.type = np.zeros(R, np.int32)
        self.rev = np.zeros(R, np.int32)
        self.nuf = np.zeros((R, K), np.int32)
        self.nur = np.zeros((R, K), np.int32)
        self.A = np.zeros(R)
        self.b = np.zeros(R)
        self.EaR = np.zeros(R)
        self.A0 = np.zeros(R)
        self.b0 = np.zeros(R)
        self.EaR0 = np.zeros(R)
        self.troe = np.zeros((R, 4))
        self.ntroe = np.zeros(R, np.int32)
        self.eff = np.ones((R, K))
        r = -1
        raw_low = {}
        while toks[pos][0] != "END":
            t = toks[pos]
            if t[0] == "RX":
                r += 1
                self.type[r] = TYPES[t[1]]
                self.rev[r] = 1 if t[2] == "REV" else 0
                q = 3
                for table in (self.nuf, self.nur):
                    nsp = int(t[q])
                    q += 1
                    for _ in range(nsp):
                        table[r, idx[t[q]]] += int(t[q + 1])
                        q += 2
                A, b, E = float(t[q]), float(t[q + 1]), float(t[q + 2])
                order = int(self.nuf[r].sum()) + (1 if self.type[r] == 1 else 0)
                self.A[r] = A * 1e-6 ** (order - 1)
                self.b[r] = b
                self.EaR[r] = E * 1e3 / RU
            elif t[0] == "EFF":
                n = int(t[1])
                for e in range(n):
                    self.eff[r, idx[t[2 + 2 * e]]] = float(t[3 + 2 * e])
            elif t[0] == "LOW":
                raw_low[r] = (float(t[1]), float(t[2]), float(t[3]))
            elif t[0] == "TROE":
                n = int(t[1])
                self.ntroe[r] = n
                vals = [float(x) for x in t[2:2 + n]]
                self.troe[r, :n] = vals
            else:
                raise ValueError("unknown record %s" % t[0])
            pos += 1
        assert r == R - 1, "reaction count mismatch"
        for rr, (A0, b0, E0) in raw_low.items():
            order = int(self.nuf[rr].sum()) + 1
            self.A0[rr] = A0 * 1e-6 ** (order - 1)
            self.b0[rr] = b0
            self.EaR0[rr] = E0 * 1e3 / RU

    def nu(self) -> np.ndarray:
        """Net stoichiometric matrix [R][K]."""
        return self.nur - self.nuf
