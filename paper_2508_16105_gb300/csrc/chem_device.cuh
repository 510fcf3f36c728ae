// Device arithmetic of the per-cell chemistry step (sm_103a, FP64).
//
// One lane integrates one cell.  All lanes of a warp run the same substep code
// on different cells, so every mechanism table read is a shared-memory
// broadcast and the FP64 pipe sees full warps.  On GB300 the FP64 pipe retires
// about two lane-operations per SM clock (measured 1.20 TFLOP/s for the GPU)
// and a warp instruction costs the same whether 1 or 32 lanes are active; the
// integer, load and select work around it is nearly free.  The design therefore
// spends integer work (index tables, selects, local memory) to save FP64
// operations and to keep all 32 lanes on useful cells.
//
// Model (Appendix A, Eqs. 20-21, closed adiabatic constant-pressure reactor):
//   c_k = rho Y_k / W_k,  rho = p / (R_u T sum_k Y_k / W_k)
//   k_f = exp(ln A + b ln T - E/(R_u T));  ln K_c = -sum_k nu_k G_k/RT + (sum nu) ln(P_std / (R_u T))
//   k_r = exp(ln k_f - ln K_c)  (reversible reactions)
//   q   = k_f prod c^nu' - k_r prod c^nu''  (times [M] for plain third-body reactions;
//         Lindemann / Troe blending k = k_inf Pr/(1+Pr) F, Pr = k_0 [M] / k_inf)
//   dY_k/dt = W_k omega_k / rho,  dT/dt = -R_u T sum_k (H/RT)_k omega_k / (rho c_p)
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "fastmath.cuh"
#include "mech_layout.h"

namespace rde {

constexpr double kRu = 8.31446261815324;        // J/(mol K)
constexpr double kLnPstdOverRu = 9.408091968943316;  // ln(101325 Pa / R_u)
constexpr double kLn10 = 2.302585092994046;

// RODAS3 (Sandu et al. 1997) in the transformed form
//   (I/(h gamma) - J) u_i = f(y + sum_j a_ij u_j) + sum_j (c_ij / h) u_j
// with gamma = 1/2; a31 = 2, a41 = 2, a43 = 1 (others 0); c21 = 4, c31 = 1,
// c32 = -1, c41 = 1, c42 = -1, c43 = -8/3; y_new = y + 2 u1 + u3 + u4; error = u4.
constexpr double kGamma = 0.5;
constexpr double kC21 = 4.0, kC31 = 1.0, kC32 = -1.0, kC41 = 1.0, kC42 = -1.0, kC43 = -8.0 / 3.0;

struct Opts {
  double rtol, atol, hmin, facmax, facmin, safety;
  int max_substeps;
  int pad;
};

// integer power for small stoichiometric orders (1..3)
__device__ __forceinline__ double ipow(double c, int e) {
  double r = c;
  if (e >= 2) r *= c;
  if (e >= 3) r *= c;
  return r;
}

// Product of c_j^order_j over one reaction side and, if dP, d(product)/d c_s for
// each listed species s.  n is uniform across the warp (same reaction in every
// lane), so the branches do not diverge and no multiplication by 1 is issued.
__device__ __forceinline__ void side_product(const int32_t* idx, const int32_t* ord, int n, const double* c,
                                             double& P, double* dP) {
  double f0 = 1.0, f1 = 1.0, f2 = 1.0;
  if (n > 0) f0 = ipow(c[idx[0]], ord[0]);
  if (n > 1) f1 = ipow(c[idx[1]], ord[1]);
  if (n > 2) f2 = ipow(c[idx[2]], ord[2]);
  P = f0;
  if (n > 1) P *= f1;
  if (n > 2) P *= f2;
  if (dP) {
    for (int s = 0; s < n; ++s) {
      const int o = ord[s];
      const double cs = c[idx[s]];
      // d(c^o)/dc = o c^(o-1)
      double d = (o == 1) ? 1.0 : (o == 2 ? 2.0 * cs : 3.0 * cs * cs);
      if (n == 2) d *= (s == 0 ? f1 : f0);
      if (n == 3) d *= (s == 0 ? f1 * f2 : (s == 1 ? f0 * f2 : f0 * f1));
      dP[s] = d;
    }
  }
}

// Per-lane temporaries of one right-hand-side evaluation.
template <int K>
struct RhsScratch {
  double c[K];     // concentrations, mol/m^3
  double g[K];     // G/RT
  double hrt[K];   // H/RT
  double cpr[K];   // Cp/R
  double wdot[K];  // net production, mol/(m^3 s)
  double wT[K];    // d wdot / dT at fixed c (Jacobian only)
};

// Troe / Lindemann blending: returns k_f and, if JAC, d ln k_f/dT (fixed [M]) and d k_f / d[M].
template <bool JAC>
__device__ __forceinline__ double falloff(const MechView& m, const RxnPacked& x, double T, double lnT, double invT,
                                          double M, double kinf, double& dlnkf, double& dkf_dM) {
  constexpr double kInvLn10 = 0.43429448190325182;
  const double k0 = exp_tab(x.lnA0 + x.b0 * lnT - x.EaR0 * invT, m.exptab);
  const double Pr = k0 * M / kinf;
  double F = 1.0, D = 0.0, dlnF_T = 0.0;
  if (x.type == RX_TROE) {
    const double e3 = exp_tab(-T * x.troe_invT3, m.exptab), e1 = exp_tab(-T * x.troe_invT1, m.exptab);
    double Fc = (1.0 - x.troe_a) * e3 + x.troe_a * e1;
    double dFc = -(1.0 - x.troe_a) * x.troe_invT3 * e3 - x.troe_a * x.troe_invT1 * e1;
    if (x.has_T2) {
      const double e2 = exp_tab(-x.troe_T2 * invT, m.exptab);
      Fc += e2;
      dFc += x.troe_T2 * invT * invT * e2;
    }
    const double Lc = log_tab(Fc, m.logtab) * kInvLn10;
    const double cc = -0.4 - 0.67 * Lc, nn = 0.75 - 1.27 * Lc, dd = 0.14;
    const double L = log_tab(fmax(Pr, 1e-300), m.logtab) * kInvLn10;
    const double u = L + cc, den = nn - dd * u, X = u / den;
    const double opx = 1.0 + X * X;
    const double logF = Lc / opx;
    F = exp_tab(kLn10 * logF, m.exptab);
    if (JAC) {
      const double dLc = dFc / (Fc * kLn10);
      const double dX_du = nn / (den * den);
      const double common = -Lc * 2.0 * X / (opx * opx);
      D = common * dX_du;
      const double du_dT = -0.67 * dLc, dn_dT = -1.27 * dLc;
      const double dX_dT = (du_dT * den - u * (dn_dT - dd * du_dT)) / (den * den);
      dlnF_T = kLn10 * (dLc / opx + common * dX_dT);
    }
  }
  const double opr = 1.0 + Pr;
  const double kf = kinf * Pr / opr * F;
  if (JAC) {
    const double dlnkinf = (x.b + x.EaR * invT) * invT;
    const double dlnk0 = (x.b0 + x.EaR0 * invT) * invT;
    const double dlnPr = dlnk0 - dlnkinf;
    dlnkf = dlnkinf + dlnF_T + D * dlnPr + dlnPr / opr;
    dkf_dM = k0 * F / opr * (D + 1.0 / opr);
  }
  return kf;
}

// f(y) and, if JAC, the Jacobian block D = d omega / d c (fixed T) accumulated into
// Mx[k*N + j] (k, j < K) plus wT = d omega / dT (fixed c).  Returns with s filled.
// y = (Y_0..Y_{K-1}, T); invp = 1/p.
template <int K, bool JAC>
__device__ __forceinline__ void eval_rhs(const MechView& m, double invp, const double* y, double* f,
                                         RhsScratch<K>& s, double* Mx, double& rho_out, double& invrho_out,
                                         double& cpm_out, double& dcpm_out, double& sumYW_out) {
  constexpr int N = K + 1;
  const double T = y[K];
  const double invT = 1.0 / T;
  const double lnT = log_tab(T, m.logtab);
  const SpecPacked* sp = m.sp;

  double sumYW = 0.0;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    s.c[k] = y[k] * sp[k].Winv;
    sumYW += s.c[k];
  }
  const double RT = kRu * T;
  const double invrho = RT * sumYW * invp;
  const double rho = 1.0 / invrho;
  double Msum = 0.0, cpm = 0.0, dcpm = 0.0;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const double yw = s.c[k];
    s.c[k] = yw * rho;
    Msum += s.c[k];
    const int r = (T >= sp[k].Tmid) ? 1 : 0;
    const double* a = sp[k].cp[r];
    const double cp = a[0] + T * (a[1] + T * (a[2] + T * (a[3] + T * a[4])));
    const double* hh = sp[k].h[r];
    const double h = hh[0] + T * (hh[1] + T * (hh[2] + T * (hh[3] + T * hh[4]))) + hh[5] * invT;
    const double* gg = sp[k].g[r];
    const double g = gg[0] + gg[1] * lnT + T * (gg[2] + T * (gg[3] + T * (gg[4] + T * gg[5]))) + gg[6] * invT;
    s.cpr[k] = cp;
    s.hrt[k] = h;
    s.g[k] = g;
    cpm += yw * cp;
    if (JAC) {
      const double* dc = sp[k].dcp[r];
      dcpm += yw * (dc[0] + T * (dc[1] + T * (dc[2] + T * dc[3])));
    }
    s.wdot[k] = 0.0;
    if (JAC) s.wT[k] = 0.0;
  }
  if (JAC) {
#pragma unroll
    for (int i = 0; i < K * N; ++i) Mx[i] = 0.0;
  }
  const double lnPRT = kLnPstdOverRu - lnT;
  const int R = m.hdr->R;
  for (int r = 0; r < R; ++r) {
    const RxnPacked& x = m.rx[r];
    const double lnk = x.lnA + x.b * lnT - x.EaR * invT;
    double M = 1.0;
    if (x.type != RX_ELEM) {
      M = Msum;
      for (int e = x.eff_begin; e < x.eff_end; ++e) M += m.eff[e].alpha_minus_1 * s.c[m.eff[e].k];
    }
    double kf, dlnkf = 0.0, dkf_dM = 0.0;
    if (x.type == RX_LINDEMANN || x.type == RX_TROE) {
      kf = falloff<JAC>(m, x, T, lnT, invT, M, exp_tab(lnk, m.exptab), dlnkf, dkf_dM);
    } else {
      kf = exp_tab(lnk, m.exptab);
      if (JAC) dlnkf = (x.b + x.EaR * invT) * invT;
    }
    double kr = 0.0, dlnKc = 0.0;
    if (x.rev) {
      // ln K_c = sum_reac nu' g - sum_prod nu'' g + dnu ln(P_std/(R_u T))
      double lnKc = x.dnu * lnPRT;
      double dh = 0.0;
      for (int q = 0; q < x.nf; ++q) {
        lnKc += x.fo[q] * s.g[x.fi[q]];
        if (JAC) dh -= x.fo[q] * s.hrt[x.fi[q]];
      }
      for (int q = 0; q < x.nb; ++q) {
        lnKc -= x.bo[q] * s.g[x.bi[q]];
        if (JAC) dh += x.bo[q] * s.hrt[x.bi[q]];
      }
      if (x.type == RX_LINDEMANN || x.type == RX_TROE) kr = kf * exp_tab(-lnKc, m.exptab);
      else kr = exp_tab(lnk - lnKc, m.exptab);
      if (JAC) dlnKc = (dh - x.dnu) * invT;
    }
    double Pf, Pb, dPf[kMaxSide], dPb[kMaxSide];
    side_product(x.fi, x.fo, x.nf, s.c, Pf, JAC ? dPf : nullptr);
    side_product(x.bi, x.bo, x.nb, s.c, Pb, JAC ? dPb : nullptr);
    const double q0 = kf * Pf - kr * Pb;
    const bool tb = (x.type == RX_THREEBODY);
    const double q = tb ? M * q0 : q0;
    for (int pp = 0; pp < x.np; ++pp) s.wdot[x.pi[pp]] += x.pnu[pp] * q;
    if (JAC) {
      const double mf = tb ? M : 1.0;
      double dqdT = kf * dlnkf * Pf - kr * (dlnkf - dlnKc) * Pb;
      dqdT *= mf;
      // term common to all species through [M]
      double allc = 0.0;
      if (tb) allc = q0;
      else if (x.type == RX_LINDEMANN || x.type == RX_TROE) allc = (kf != 0.0) ? dkf_dM * (q0 / kf) : 0.0;
      for (int pp = 0; pp < x.np; ++pp) {
        const int k = x.pi[pp];
        const double nu = x.pnu[pp];
        s.wT[k] += nu * dqdT;
        double* row = Mx + k * N;
        for (int q1 = 0; q1 < x.nf; ++q1) row[x.fi[q1]] += nu * mf * kf * dPf[q1];
        for (int q1 = 0; q1 < x.nb; ++q1) row[x.bi[q1]] -= nu * mf * kr * dPb[q1];
        if (x.type != RX_ELEM) {
          const double base = nu * allc;
#pragma unroll
          for (int j = 0; j < K; ++j) row[j] += base;
          for (int e = x.eff_begin; e < x.eff_end; ++e) row[m.eff[e].k] += base * m.eff[e].alpha_minus_1;
        }
      }
    }
  }
  // f
  double sum_hw = 0.0;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    f[k] = sp[k].W * s.wdot[k] * invrho;
    sum_hw += s.hrt[k] * s.wdot[k];
  }
  const double cpm_J = kRu * cpm;  // J/(kg K)
  f[K] = -RT * sum_hw * invrho / cpm_J;
  rho_out = rho;
  invrho_out = invrho;
  cpm_out = cpm_J;
  dcpm_out = kRu * dcpm;
  sumYW_out = sumYW;
}

// Complete the Jacobian from D (in Mx[0..K)[0..K)), then store M = I/(gamma h) - J in Mx.
template <int K>
__device__ __forceinline__ void assemble_matrix(const MechView& m, const double* y, const double* f,
                                                const RhsScratch<K>& s, double rho, double invrho, double cpm,
                                                double dcpm, double sumYW, double inv_gh, double* Mx, double* Dc,
                                                double* HD) {
  constexpr int N = K + 1;
  const double T = y[K];
  const double invT = 1.0 / T;
  const double RT = kRu * T;
  const double Wbar = 1.0 / sumYW;
  const SpecPacked* sp = m.sp;
  double HDc = 0.0, Cw = 0.0, HwT = 0.0;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    double acc = 0.0;
#pragma unroll
    for (int j = 0; j < K; ++j) acc += Mx[k * N + j] * s.c[j];
    Dc[k] = acc;
  }
#pragma unroll
  for (int i = 0; i < K; ++i) {
    double acc = 0.0;
#pragma unroll
    for (int k = 0; k < K; ++k) acc += s.hrt[k] * Mx[k * N + i];
    HD[i] = acc;
  }
#pragma unroll
  for (int k = 0; k < K; ++k) {
    HDc += s.hrt[k] * Dc[k];
    Cw += s.cpr[k] * s.wdot[k];
    HwT += s.hrt[k] * (s.wT[k] - Dc[k] * invT);
  }
  const double fT = f[K];
  // species rows: J_ki = W_k/W_i D_ki + W_k Wbar/(W_i rho) (wdot_k - Dc_k);  J_kT
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const double Wk = sp[k].W;
    const double Bk = Wk * Wbar * (s.wdot[k] - Dc[k]) * invrho;
#pragma unroll
    for (int i = 0; i < K; ++i) {
      const double J = sp[i].Winv * (Wk * Mx[k * N + i] + Bk);
      Mx[k * N + i] = (i == k ? inv_gh : 0.0) - J;
    }
    const double JkT = Wk * invrho * (s.wT[k] + (s.wdot[k] - Dc[k]) * invT);
    Mx[k * N + K] = -JkT;
  }
  // temperature row
  const double inv_cp = 1.0 / cpm;
  const double coef = -RT * inv_cp;
#pragma unroll
  for (int i = 0; i < K; ++i) {
    const double J = coef * sp[i].Winv * (HD[i] - Wbar * invrho * HDc) -
                     fT * sp[i].Winv * (kRu * s.cpr[i] - cpm * Wbar) * inv_cp;
    Mx[K * N + i] = -J;
  }
  const double JTT = -(kRu * Cw + RT * HwT) * invrho * inv_cp + fT * invT - fT * dcpm * inv_cp;
  Mx[K * N + K] = inv_gh - JTT;
  (void)rho;
}

// In-place LU with partial pivoting (row-major N x N); stores 1/U_kk in invd.
// Returns false on a zero pivot.
template <int N>
__device__ __forceinline__ bool lu_factor(double* Mx, int* piv, double* invd) {
  bool ok = true;
#pragma unroll
  for (int k = 0; k < N; ++k) {
    int p = k;
    double amax = fabs(Mx[k * N + k]);
#pragma unroll
    for (int i = k + 1; i < N; ++i) {
      const double v = fabs(Mx[i * N + k]);
      if (v > amax) { amax = v; p = i; }
    }
    piv[k] = p;
    if (amax == 0.0) ok = false;
    if (p != k) {
#pragma unroll
      for (int j = 0; j < N; ++j) {
        const double t = Mx[k * N + j];
        Mx[k * N + j] = Mx[p * N + j];
        Mx[p * N + j] = t;
      }
    }
    const double inv = 1.0 / Mx[k * N + k];
    invd[k] = inv;
#pragma unroll
    for (int i = k + 1; i < N; ++i) {
      const double l = Mx[i * N + k] * inv;
      Mx[i * N + k] = l;
#pragma unroll
      for (int j = k + 1; j < N; ++j) Mx[i * N + j] -= l * Mx[k * N + j];
    }
  }
  return ok;
}

// Solve (LU) x = b in place; the row interchanges are applied with selects so b stays in registers.
template <int N>
__device__ __forceinline__ void lu_solve(const double* Mx, const int* piv, const double* invd, double* b) {
#pragma unroll
  for (int k = 0; k < N; ++k) {
    const int p = piv[k];
#pragma unroll
    for (int i = k + 1; i < N; ++i) {
      const bool sw = (p == i);
      const double bk = b[k], bi = b[i];
      b[k] = sw ? bi : bk;
      b[i] = sw ? bk : bi;
    }
  }
#pragma unroll
  for (int i = 1; i < N; ++i) {
    double acc = b[i];
#pragma unroll
    for (int j = 0; j < i; ++j) acc -= Mx[i * N + j] * b[j];
    b[i] = acc;
  }
#pragma unroll
  for (int i = N - 1; i >= 0; --i) {
    double acc = b[i];
#pragma unroll
    for (int j = i + 1; j < N; ++j) acc -= Mx[i * N + j] * b[j];
    b[i] = acc * invd[i];
  }
}

}  // namespace rde
