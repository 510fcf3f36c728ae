// Discrete adjoint of the per-cell chemistry step (sm_103a, FP64): device code,
// templated on the reaction sequence (generic or specialised to a mechanism).
//
// Differentiates the map (T0, Y0, ln A_r, E_r) -> (T, Y)(dt) along each cell's
// frozen sequence of accepted RODAS3 steps (the step sizes are held fixed; the
// rejected attempts and the controller contribute nothing).  Three kernels:
//
//  1. record:  the forward integration again, writing the start state y_n and
//              the size h_n of every accepted step into a pool at per-cell
//              offsets (an exclusive scan of the forward pass's step counts)
//              and, when the caller's workspace holds them, the step's stage
//              checkpoint: the LU factors of M and the stage vectors u_1..u_4;
//  2. reverse: a persistent queue over cells; each lane walks its cell's steps
//              backwards.  Per step it reads the stage checkpoint or recomputes
//              the stages (J(y_n), the LU of M = I/(gamma h) - J, u_1..u_4),
//              then propagates the cotangent:
//                  w_i = M^-T ubar_i                       (transposed LU solves)
//                  ybar += J(Y_i)^T w_i,  ubar_j += a_ij J(Y_i)^T w_i + c_ij/h w_i
//                  ybar += grad_y (w_i^T J(y) u_i),  thbar += grad_th (w_i^T J u_i)
//              J^T w is contracted on the fly (no matrix is formed), and the
//              second-derivative terms grad(w^T J u) = d/de [J(y + e u)^T w] come
//              from one dual-number evaluation of that contraction per stage;
//  3. reduce:  per-cell parameter gradients summed over cells in a fixed order
//              (bitwise reproducible; no floating-point atomics).
//
// Parameters: ln A_r (of k_inf for falloff reactions) and E_r in J/mol.
#pragma once
#if !defined(__CUDACC_RTC__)  /* run-time compilation: types from the preamble */
#include <cuda_runtime.h>
#include <stdint.h>
#endif

#include "chem_device.cuh"
#include "chem_launch.h"
#include "dual_math.cuh"

namespace rde {

constexpr unsigned kFullA = 0xffffffffu;
constexpr int kThreadsA = kLaneThreads;

// lane-slot view of an array of S (a Dual takes two slots)
template <class S>
struct SArr;
template <>
struct SArr<double> {
  Lane L;
  int base;
  __device__ __forceinline__ double get(int i) const { return L[base + i]; }
  __device__ __forceinline__ void set(int i, double v) const { L[base + i] = v; }
  __device__ __forceinline__ void add(int i, double v) const { L[base + i] += v; }
};
template <>
struct SArr<Dual> {
  Lane L;
  int base;
  __device__ __forceinline__ Dual get(int i) const { return mk(L[base + 2 * i], L[base + 2 * i + 1]); }
  __device__ __forceinline__ void set(int i, Dual v) const {
    L[base + 2 * i] = v.v;
    L[base + 2 * i + 1] = v.d;
  }
  __device__ __forceinline__ void add(int i, Dual v) const {
    L[base + 2 * i] += v.v;
    L[base + 2 * i + 1] += v.d;
  }
};

// Slot map of the reverse kernel.  The forward slots keep the forward kernel's
// names (so eval_rhs / assemble_matrix serve both); pivots live in a register
// and 1/U_kk replaces U_kk on the diagonal.  The nine species arrays of the
// primal J^T w contraction (c, G/RT, H/RT, Cp/R, wdot, dwdot/dT, sum wt D,
// sum H D, D c) are contiguous from C.  In the second-derivative phase, when
// the LU is no longer needed, nine dual arrays of K (18 K slots) start at 0.
template <int K>
struct AdjSlots {
  static constexpr int N = K + 1;
  static constexpr int MX = 0;
  static constexpr int C = MX + N * N;
  static constexpr int G = C + K;
  static constexpr int HRT = G + K;
  static constexpr int CPR = HRT + K;
  static constexpr int WDOT = CPR + K;
  static constexpr int WT = WDOT + K;
  static constexpr int WD = WT + K;
  static constexpr int HD = WD + K;
  static constexpr int DC = HD + K;
  static constexpr int ARG = (DC + K > 18 * K) ? DC + K : 18 * K;   // room for the dual arrays
  static constexpr int VEC = ARG + N;
  static constexpr int TOTAL = VEC + N;
  static constexpr size_t bytes(int threads) { return sizeof(double) * TOTAL * threads; }
};

// ---------------------------------------------------------------------------
// LU with the pivots in a 4-bit-per-row register word and 1/U_kk on the diagonal
// ---------------------------------------------------------------------------
template <int K>
__device__ __forceinline__ bool lu_factor_r(Lane L, unsigned long long& piv) {
  using S = AdjSlots<K>;
  constexpr int N = S::N;
  static_assert(N <= 16, "pivot word holds 16 rows");
  bool ok = true;
  piv = 0ull;
#pragma unroll 1
  for (int k = 0; k < N; ++k) {
    int p = k;
    double amax = fabs(L[S::MX + k * N + k]);
    for (int i = k + 1; i < N; ++i) {
      const double v = fabs(L[S::MX + i * N + k]);
      if (v > amax) {
        amax = v;
        p = i;
      }
    }
    piv |= (unsigned long long)p << (4 * k);
    if (amax == 0.0) ok = false;
    if (p != k) {
#pragma unroll 2
      for (int j = 0; j < N; ++j) {
        const double t = L[S::MX + k * N + j];
        L[S::MX + k * N + j] = L[S::MX + p * N + j];
        L[S::MX + p * N + j] = t;
      }
    }
    const double inv = 1.0 / L[S::MX + k * N + k];
    L[S::MX + k * N + k] = inv;
#pragma unroll 1
    for (int i = k + 1; i < N; ++i) {
      const double l = L[S::MX + i * N + k] * inv;
      L[S::MX + i * N + k] = l;
#pragma unroll 3
      for (int j = k + 1; j < N; ++j) L[S::MX + i * N + j] -= l * L[S::MX + k * N + j];
    }
  }
  return ok;
}

// M x = b in place in VEC
template <int K>
__device__ __forceinline__ void lu_solve_r(Lane L, unsigned long long piv) {
  using S = AdjSlots<K>;
  constexpr int N = S::N;
#pragma unroll 1
  for (int k = 0; k < N; ++k) {
    const int p = (int)((piv >> (4 * k)) & 15ull);
    if (p != k) {
      const double t = L[S::VEC + k];
      L[S::VEC + k] = L[S::VEC + p];
      L[S::VEC + p] = t;
    }
  }
#pragma unroll 1
  for (int i = 1; i < N; ++i) {
    double acc = L[S::VEC + i];
#pragma unroll 3
    for (int j = 0; j < i; ++j) acc -= L[S::MX + i * N + j] * L[S::VEC + j];
    L[S::VEC + i] = acc;
  }
#pragma unroll 1
  for (int i = N - 1; i >= 0; --i) {
    double acc = L[S::VEC + i];
#pragma unroll 3
    for (int j = i + 1; j < N; ++j) acc -= L[S::MX + i * N + j] * L[S::VEC + j];
    L[S::VEC + i] = acc * L[S::MX + i * N + i];
  }
}

// M^T x = b in place in VEC: P M = L U, so M^T = U^T L^T P; solve U^T z = b,
// L^T v = z, then undo the row interchanges in reverse order.
template <int K>
__device__ __forceinline__ void lu_solve_t(Lane L, unsigned long long piv) {
  using S = AdjSlots<K>;
  constexpr int N = S::N;
#pragma unroll 1
  for (int i = 0; i < N; ++i) {
    double acc = L[S::VEC + i];
#pragma unroll 3
    for (int j = 0; j < i; ++j) acc -= L[S::MX + j * N + i] * L[S::VEC + j];
    L[S::VEC + i] = acc * L[S::MX + i * N + i];
  }
#pragma unroll 1
  for (int i = N - 2; i >= 0; --i) {
    double acc = L[S::VEC + i];
#pragma unroll 3
    for (int j = i + 1; j < N; ++j) acc -= L[S::MX + j * N + i] * L[S::VEC + j];
    L[S::VEC + i] = acc;
  }
#pragma unroll 1
  for (int k = N - 1; k >= 0; --k) {
    const int p = (int)((piv >> (4 * k)) & 15ull);
    if (p != k) {
      const double t = L[S::VEC + k];
      L[S::VEC + k] = L[S::VEC + p];
      L[S::VEC + p] = t;
    }
  }
}

// ---------------------------------------------------------------------------
// J^T w without forming J, and the parameter cotangents, at state y (of type S)
// ---------------------------------------------------------------------------

// g = J(y)^T w (value, or derivative part for S = Dual), with the parameter
// cotangents w^T df/d(ln A_r) and w^T df/dE_r (value or derivative part) added
// to the lane's global accumulators thA[r * stride], thE[r * stride].
// y: N values of S; w: N primal values.  Uses slots from `base` (arrays of S).
template <int K, class S, class RX>
__device__ void jtw(const MechView& m, Lane L, int base, double invp, const S* y, const double* w, double* g,
                    double* thA, double* thE, long long stride) {
  constexpr int N = K + 1;
  constexpr int ES = sizeof(S) / sizeof(double);
  const SArr<S> Cc{L, base + 0 * ES * K}, Gg{L, base + 1 * ES * K}, Hh{L, base + 2 * ES * K},
      Cp{L, base + 3 * ES * K}, Wd{L, base + 4 * ES * K}, Wt{L, base + 5 * ES * K}, WDv{L, base + 6 * ES * K},
      HDv{L, base + 7 * ES * K}, DCv{L, base + 8 * ES * K};
  const SpecPacked* sp = m.sp;
  const S T = y[K];
  const S invT = 1.0 / T;
  const S lnT = slog(m, T);
  S sumYW = cst<S>(0.0);
#pragma unroll
  for (int k = 0; k < K; ++k) sumYW += y[k] * sp[k].Winv;
  const S RT = kRu * T;
  const S invrho = RT * sumYW * invp;
  const S rho = 1.0 / invrho;
  S Msum = cst<S>(0.0), cpm = cst<S>(0.0), dcpm = cst<S>(0.0);
#pragma unroll 1
  for (int k = 0; k < K; ++k) {
    const S yw = y[k] * sp[k].Winv;
    const S c = yw * rho;
    Cc.set(k, c);
    Msum += c;
    const int r = (val(T) >= sp[k].Tmid) ? 1 : 0;
    const double* a = sp[k].cp[r];
    const S cp = a[0] + T * (a[1] + T * (a[2] + T * (a[3] + T * a[4])));
    const double* hh = sp[k].h[r];
    const S h = hh[0] + T * (hh[1] + T * (hh[2] + T * (hh[3] + T * hh[4]))) + hh[5] * invT;
    const double* gg = sp[k].g[r];
    const S gv = gg[0] + gg[1] * lnT + T * (gg[2] + T * (gg[3] + T * (gg[4] + T * gg[5]))) + gg[6] * invT;
    const double* dc = sp[k].dcp[r];
    dcpm += yw * (dc[0] + T * (dc[1] + T * (dc[2] + T * dc[3])));
    cpm += yw * cp;
    Gg.set(k, gv);
    Hh.set(k, h);
    Cp.set(k, cp);
    Wd.set(k, cst<S>(0.0));
    Wt.set(k, cst<S>(0.0));
    WDv.set(k, cst<S>(0.0));
    HDv.set(k, cst<S>(0.0));
    DCv.set(k, cst<S>(0.0));
  }
  const S cpm_J = kRu * cpm;
  const S lnPRT = kLnPstdOverRu - lnT;
  const S fac_T = (w[K] * RT) / cpm_J;   // weight of the temperature row in w^T df/dq
  RX::each(m, [&](const auto& x, int r) {
    const S lnk = x.lnA() + x.b() * lnT - x.EaR() * invT;
    S M = cst<S>(1.0);
    if (x.type() != RX_ELEM) {
      M = Msum;
      for (int e = x.eff_begin(); e < x.eff_end(); ++e) M += x.eff_am1(m, e) * Cc.get(x.eff_k(m, e));
    }
    const bool fo = (x.type() == RX_LINDEMANN || x.type() == RX_TROE);
    S kf, dlnkf, dkf_dM = cst<S>(0.0), phi = cst<S>(1.0);
    if (fo) {
      kf = falloff_s<S>(m, x, T, lnT, invT, M, sexp(m, lnk), dlnkf, dkf_dM, phi);
    } else {
      kf = sexp(m, lnk);
      dlnkf = (x.b() + x.EaR() * invT) * invT;
    }
    S kr = cst<S>(0.0), dlnKc = cst<S>(0.0);
    if (x.rev()) {
      S lnKc = x.dnu() * lnPRT;
      S dh = cst<S>(0.0);
      for (int q = 0; q < x.nf(); ++q) {
        lnKc += x.fod(q) * Gg.get(x.fi(q));
        dh -= x.fod(q) * Hh.get(x.fi(q));
      }
      for (int q = 0; q < x.nb(); ++q) {
        lnKc -= x.bod(q) * Gg.get(x.bi(q));
        dh += x.bod(q) * Hh.get(x.bi(q));
      }
      kr = fo ? kf * sexp(m, -lnKc) : sexp(m, lnk - lnKc);
      dlnKc = (dh - x.dnu()) * invT;
    }
    S cf[kMaxSide], cb[kMaxSide], pf[kMaxSide], pb[kMaxSide];
#pragma unroll
    for (int q = 0; q < kMaxSide; ++q) {
      cf[q] = (q < x.nf()) ? Cc.get(x.fi(q)) : cst<S>(1.0);
      cb[q] = (q < x.nb()) ? Cc.get(x.bi(q)) : cst<S>(1.0);
      pf[q] = (q < x.nf()) ? ipow_s(cf[q], x.fo(q)) : cst<S>(1.0);
      pb[q] = (q < x.nb()) ? ipow_s(cb[q], x.bo(q)) : cst<S>(1.0);
    }
    S Pf = pf[0], Pb = pb[0];
    if (x.nf() > 1) Pf = Pf * pf[1];
    if (x.nf() > 2) Pf = Pf * pf[2];
    if (x.nb() > 1) Pb = Pb * pb[1];
    if (x.nb() > 2) Pb = Pb * pb[2];
    const S q0 = kf * Pf - kr * Pb;
    const bool tb = (x.type() == RX_THREEBODY);
    const S mf = tb ? M : cst<S>(1.0);
    const S q = mf * q0;
    const S dqdT = mf * (kf * dlnkf * Pf - kr * (dlnkf - dlnKc) * Pb);
    // contraction weights of this reaction: s1 = sum_p wt_p nu_p, s2 = sum_p (H/RT)_p nu_p
    double s1 = 0.0;
    S s2 = cst<S>(0.0);
    for (int pp = 0; pp < x.np(); ++pp) {
      const int k = x.pi(pp);
      s1 += w[k] * sp[k].W * x.pnu(pp);
      s2 += x.pnu(pp) * Hh.get(k);
    }
    // gradient of q w.r.t. the concentrations of each side's species, and grad q . c
    S gf[kMaxSide], gb[kMaxSide];
    const S mkf = mf * kf, mkr = mf * kr;
    S gc = cst<S>(0.0);
#pragma unroll
    for (int s = 0; s < kMaxSide; ++s) {
      const S df = (x.fo(s) == 1) ? cst<S>(1.0) : (x.fo(s) == 2 ? 2.0 * cf[s] : 3.0 * (cf[s] * cf[s]));
      const S db = (x.bo(s) == 1) ? cst<S>(1.0) : (x.bo(s) == 2 ? 2.0 * cb[s] : 3.0 * (cb[s] * cb[s]));
      S of = cst<S>(1.0), ob = cst<S>(1.0);
#pragma unroll
      for (int t = 0; t < kMaxSide; ++t) {
        if (t != s && t < x.nf()) of = of * pf[t];
        if (t != s && t < x.nb()) ob = ob * pb[t];
      }
      gf[s] = mkf * df * of;
      gb[s] = -(mkr * db * ob);
      if (s < x.nf()) gc += gf[s] * cf[s];
      if (s < x.nb()) gc += gb[s] * cb[s];
    }
    S allc = cst<S>(0.0);
    if (tb) allc = q0;
    else if (fo) allc = (val(kf) != 0.0) ? dkf_dM * (q0 / kf) : cst<S>(0.0);
    if (x.type() != RX_ELEM) gc += allc * M;
    for (int pp = 0; pp < x.np(); ++pp) {
      const int k = x.pi(pp);
      const double nu = x.pnu(pp);
      Wd.add(k, nu * q);
      Wt.add(k, nu * dqdT);
      DCv.add(k, nu * gc);
    }
    for (int s = 0; s < x.nf(); ++s) {
      WDv.add(x.fi(s), s1 * gf[s]);
      HDv.add(x.fi(s), s2 * gf[s]);
    }
    for (int s = 0; s < x.nb(); ++s) {
      WDv.add(x.bi(s), s1 * gb[s]);
      HDv.add(x.bi(s), s2 * gb[s]);
    }
    if (x.type() != RX_ELEM) {
      const S a1 = s1 * allc, a2 = s2 * allc;
#pragma unroll 1
      for (int j = 0; j < K; ++j) {
        WDv.add(j, a1);
        HDv.add(j, a2);
      }
      for (int e = x.eff_begin(); e < x.eff_end(); ++e) {
        WDv.add(x.eff_k(m, e), a1 * x.eff_am1(m, e));
        HDv.add(x.eff_k(m, e), a2 * x.eff_am1(m, e));
      }
    }
    // w^T df/dq_r = (s1 - w_T R T s2 / c_p) / rho;  d q / d ln A = phi q;  d q / d E = -phi q / (R T)
    const S sr = (s1 - fac_T * s2) * invrho;
    const S tA = sr * phi * q;
    const S tE = -(tA / RT);
    thA[r * stride] += (ES == 1) ? val(tA) : der(tA);
    thE[r * stride] += (ES == 1) ? val(tE) : der(tE);
  });
  // f_T and the assembly of J^T w
  S sum_hw = cst<S>(0.0), wfe = cst<S>(0.0), wfT = cst<S>(0.0), HDc = cst<S>(0.0), Cw = cst<S>(0.0),
    HwT = cst<S>(0.0);
#pragma unroll 1
  for (int k = 0; k < K; ++k) {
    const S wd = Wd.get(k), dc = DCv.get(k), h = Hh.get(k), wt = Wt.get(k);
    const double wtk = w[k] * sp[k].W;
    sum_hw += h * wd;
    wfe += wtk * (wd - dc);
    wfT += wtk * (wt + (wd - dc) * invT);
    HDc += h * dc;
    Cw += Cp.get(k) * wd;
    HwT += h * (wt - dc * invT);
  }
  const S fT = -(RT * sum_hw * invrho) / cpm_J;
  const S Wbar = 1.0 / sumYW;
  const S beta = Wbar * invrho * wfe;
  const S inv_cp = 1.0 / cpm_J;
  const S coef = -(RT * inv_cp);
  const S wHDc = Wbar * invrho * HDc;
  const S fcp = fT * inv_cp;
#pragma unroll 1
  for (int i = 0; i < K; ++i) {
    const S gi = sp[i].Winv * (WDv.get(i) + beta +
                               w[K] * (coef * (HDv.get(i) - wHDc) - fcp * (kRu * Cp.get(i) - cpm_J * Wbar)));
    g[i] = (ES == 1) ? val(gi) : der(gi);
  }
  const S JTT = -((kRu * Cw + RT * HwT) * invrho * inv_cp) + fT * invT - fT * (kRu * dcpm) * inv_cp;
  const S gT = invrho * wfT + w[K] * JTT;
  g[K] = (ES == 1) ? val(gT) : der(gT);
}

// ---------------------------------------------------------------------------
// Second-derivative terms of several stages in one evaluation
// ---------------------------------------------------------------------------
// A value with ND derivative parts (directions).  The stage terms
//     ybar += sum_i grad_y (w_i^T J(y) u_i)
// share the point y, so one evaluation can carry ND directions u_i: the primal
// part (rates, exponentials, thermo) is computed once instead of once per
// direction.  The species accumulators of jtw keep only their primal parts,
// which do not depend on w; their derivative parts are contracted with the
// weights of the final assembly as they are added, into per-direction scalars
// and two direction-summed species arrays.
template <int ND>
struct DualN {
  double v;
  double d[ND];
};
template <int ND>
__device__ __forceinline__ DualN<ND> dn_const(double v) {
  DualN<ND> r;
  r.v = v;
#pragma unroll
  for (int i = 0; i < ND; ++i) r.d[i] = 0.0;
  return r;
}
template <int ND>
__device__ __forceinline__ DualN<ND> operator+(const DualN<ND>& a, const DualN<ND>& b) {
  DualN<ND> r;
  r.v = a.v + b.v;
#pragma unroll
  for (int i = 0; i < ND; ++i) r.d[i] = a.d[i] + b.d[i];
  return r;
}
template <int ND>
__device__ __forceinline__ DualN<ND> operator-(const DualN<ND>& a, const DualN<ND>& b) {
  DualN<ND> r;
  r.v = a.v - b.v;
#pragma unroll
  for (int i = 0; i < ND; ++i) r.d[i] = a.d[i] - b.d[i];
  return r;
}
template <int ND>
__device__ __forceinline__ DualN<ND> operator-(const DualN<ND>& a) {
  DualN<ND> r;
  r.v = -a.v;
#pragma unroll
  for (int i = 0; i < ND; ++i) r.d[i] = -a.d[i];
  return r;
}
template <int ND>
__device__ __forceinline__ DualN<ND> operator+(const DualN<ND>& a, double b) {
  DualN<ND> r = a;
  r.v = a.v + b;
  return r;
}
template <int ND>
__device__ __forceinline__ DualN<ND> operator+(double a, const DualN<ND>& b) { return b + a; }
template <int ND>
__device__ __forceinline__ DualN<ND> operator-(const DualN<ND>& a, double b) {
  DualN<ND> r = a;
  r.v = a.v - b;
  return r;
}
template <int ND>
__device__ __forceinline__ DualN<ND> operator-(double a, const DualN<ND>& b) {
  DualN<ND> r;
  r.v = a - b.v;
#pragma unroll
  for (int i = 0; i < ND; ++i) r.d[i] = -b.d[i];
  return r;
}
template <int ND>
__device__ __forceinline__ DualN<ND> operator*(const DualN<ND>& a, const DualN<ND>& b) {
  DualN<ND> r;
  r.v = a.v * b.v;
#pragma unroll
  for (int i = 0; i < ND; ++i) r.d[i] = fma(a.v, b.d[i], a.d[i] * b.v);
  return r;
}
template <int ND>
__device__ __forceinline__ DualN<ND> operator*(double a, const DualN<ND>& b) {
  DualN<ND> r;
  r.v = a * b.v;
#pragma unroll
  for (int i = 0; i < ND; ++i) r.d[i] = a * b.d[i];
  return r;
}
template <int ND>
__device__ __forceinline__ DualN<ND> operator*(const DualN<ND>& a, double b) { return b * a; }
template <int ND>
__device__ __forceinline__ DualN<ND> operator/(const DualN<ND>& a, const DualN<ND>& b) {
  const double inv = 1.0 / b.v;
  DualN<ND> r;
  r.v = a.v * inv;
#pragma unroll
  for (int i = 0; i < ND; ++i) r.d[i] = (a.d[i] - r.v * b.d[i]) * inv;
  return r;
}
template <int ND>
__device__ __forceinline__ DualN<ND> operator/(double a, const DualN<ND>& b) {
  const double inv = 1.0 / b.v;
  DualN<ND> r;
  r.v = a * inv;
#pragma unroll
  for (int i = 0; i < ND; ++i) r.d[i] = -(r.v * b.d[i]) * inv;
  return r;
}
template <int ND>
__device__ __forceinline__ DualN<ND> operator/(const DualN<ND>& a, double b) {
  DualN<ND> r;
  r.v = a.v / b;
#pragma unroll
  for (int i = 0; i < ND; ++i) r.d[i] = a.d[i] / b;
  return r;
}
template <int ND>
__device__ __forceinline__ DualN<ND>& operator+=(DualN<ND>& a, const DualN<ND>& b) { a = a + b; return a; }
template <int ND>
__device__ __forceinline__ DualN<ND>& operator-=(DualN<ND>& a, const DualN<ND>& b) { a = a - b; return a; }
template <int ND>
__device__ __forceinline__ DualN<ND>& operator*=(DualN<ND>& a, const DualN<ND>& b) { a = a * b; return a; }
template <int ND>
__device__ __forceinline__ double val(const DualN<ND>& x) { return x.v; }
template <> __device__ __forceinline__ DualN<2> cst<DualN<2>>(double v) { return dn_const<2>(v); }
template <> __device__ __forceinline__ DualN<4> cst<DualN<4>>(double v) { return dn_const<4>(v); }
template <int ND>
__device__ __forceinline__ DualN<ND> sexp(const MechView& m, const DualN<ND>& x) {
  const double e = exp_tab(x.v, m.exptab);
  DualN<ND> r;
  r.v = e;
#pragma unroll
  for (int i = 0; i < ND; ++i) r.d[i] = e * x.d[i];
  return r;
}
template <int ND>
__device__ __forceinline__ DualN<ND> slog(const MechView& m, const DualN<ND>& x) {
  DualN<ND> r;
  r.v = log_tab(x.v, m.logtab);
#pragma unroll
  for (int i = 0; i < ND; ++i) r.d[i] = x.d[i] / x.v;
  return r;
}
template <int ND>
__device__ __forceinline__ DualN<ND> smax300(const DualN<ND>& x) { return x.v > 1e-300 ? x : dn_const<ND>(1e-300); }
// direction i of x as a single dual number
template <int ND>
__device__ __forceinline__ Dual view(const DualN<ND>& x, int i) { return mk(x.v, x.d[i]); }

// Slots of hvp_sum (arrays of K from 0): concentrations and their ND derivative
// parts; G/RT, H/RT, Cp/R and their temperature derivatives; the primal
// accumulators (production, its T-derivative, D c, sum H D); the direction-
// summed derivative parts of sum w D and of w_T sum H D.
template <int K, int ND>
struct HvpSlots {
  static constexpr int C = 0, CD = C + K, GV = CD + ND * K, GD = GV + K, HV = GD + K, HD = HV + K, PV = HD + K,
                       PD = PV + K, WDP = PD + K, WTP = WDP + K, DCP = WTP + K, HDP = DCP + K, WDS = HDP + K,
                       HDS = WDS + K, TOTAL = HDS + K;
};

// g += sum_{i < ND} d/de [J(y + e u_i)^T w_i] and the parameter terms
// d/de [w_i^T df/d(ln A_r)], d/de [w_i^T df/dE_r] added to thA / thE.  y: N primal
// values; u_i, w_i: stages st0 .. st0 + ND - 1 of the lane's U and W (element e
// of stage s at [(s N + e) nl]).  Each direction's terms equal those of one
// dual-number evaluation of jtw, up to rounding order.
template <int K, int ND, class RX>
__device__ __forceinline__ void hvp_sum(const MechView& m, Lane L, double invp, const double* y, const double* U,
                                        const double* W, int st0, long long nl, double* g, double* thA, double* thE,
                                        long long stride) {
  constexpr int N = K + 1;
  using D = DualN<ND>;
  using HS = HvpSlots<K, ND>;
  static_assert(HS::TOTAL <= 18 * K, "hvp_sum slots exceed the reverse kernel's dual area");
  const SpecPacked* sp = m.sp;
  auto u_at = [&](int i, int e) { return U[((long long)(st0 + i) * N + e) * nl]; };
  auto w_at = [&](int i, int e) { return W[((long long)(st0 + i) * N + e) * nl]; };
  double wK[ND];
  D T;
  T.v = y[K];
#pragma unroll
  for (int i = 0; i < ND; ++i) {
    T.d[i] = u_at(i, K);
    wK[i] = w_at(i, K);
  }
  const D invT = 1.0 / T;
  const D lnT = slog(m, T);
  // temperature polynomials carry a unit derivative: X and dX/dT
  const Dual Tu = mk(y[K], 1.0);
  const Dual invTu = 1.0 / Tu;
  const Dual lnTu = slog(m, Tu);
  D sumYW = cst<D>(0.0);
#pragma unroll
  for (int k = 0; k < K; ++k) {
    D yw;
    yw.v = y[k] * sp[k].Winv;
#pragma unroll
    for (int i = 0; i < ND; ++i) yw.d[i] = u_at(i, k) * sp[k].Winv;
    sumYW += yw;
  }
  const D RT = kRu * T;
  const D invrho = RT * sumYW * invp;
  const D rho = 1.0 / invrho;
  D Msum = cst<D>(0.0), cpm = cst<D>(0.0), dcpm = cst<D>(0.0);
#pragma unroll
  for (int k = 0; k < K; ++k) {
    D yw;
    yw.v = y[k] * sp[k].Winv;
#pragma unroll
    for (int i = 0; i < ND; ++i) yw.d[i] = u_at(i, k) * sp[k].Winv;
    const D c = yw * rho;
    L[HS::C + k] = c.v;
#pragma unroll
    for (int i = 0; i < ND; ++i) L[HS::CD + i * K + k] = c.d[i];
    Msum += c;
    const int r = (y[K] >= sp[k].Tmid) ? 1 : 0;
    const double* a = sp[k].cp[r];
    const Dual cp = a[0] + Tu * (a[1] + Tu * (a[2] + Tu * (a[3] + Tu * a[4])));
    const double* hh = sp[k].h[r];
    const Dual h = hh[0] + Tu * (hh[1] + Tu * (hh[2] + Tu * (hh[3] + Tu * hh[4]))) + hh[5] * invTu;
    const double* gg = sp[k].g[r];
    const Dual gv = gg[0] + gg[1] * lnTu + Tu * (gg[2] + Tu * (gg[3] + Tu * (gg[4] + Tu * gg[5]))) + gg[6] * invTu;
    const double* dc = sp[k].dcp[r];
    dcpm += yw * (dc[0] + T * (dc[1] + T * (dc[2] + T * dc[3])));
    D cpn;
    cpn.v = cp.v;
#pragma unroll
    for (int i = 0; i < ND; ++i) cpn.d[i] = cp.d * T.d[i];
    cpm += yw * cpn;
    L[HS::GV + k] = gv.v;
    L[HS::GD + k] = gv.d;
    L[HS::HV + k] = h.v;
    L[HS::HD + k] = h.d;
    L[HS::PV + k] = cp.v;
    L[HS::PD + k] = cp.d;
    L[HS::WDP + k] = 0.0;
    L[HS::WTP + k] = 0.0;
    L[HS::DCP + k] = 0.0;
    L[HS::HDP + k] = 0.0;
    L[HS::WDS + k] = 0.0;
    L[HS::HDS + k] = 0.0;
  }
  auto cget = [&](int k) {
    D r;
    r.v = L[HS::C + k];
#pragma unroll
    for (int i = 0; i < ND; ++i) r.d[i] = L[HS::CD + i * K + k];
    return r;
  };
  auto tget = [&](int vbase, int dbase, int k) {
    D r;
    r.v = L[vbase + k];
    const double dd = L[dbase + k];
#pragma unroll
    for (int i = 0; i < ND; ++i) r.d[i] = dd * T.d[i];
    return r;
  };
  const D cpm_J = kRu * cpm;
  const D lnPRT = kLnPstdOverRu - lnT;
  Dual facT[ND];   // weight of the temperature row in w_i^T df/dq, direction i
#pragma unroll
  for (int i = 0; i < ND; ++i) facT[i] = (wK[i] * view(RT, i)) / view(cpm_J, i);
  // derivative parts already contracted with the final assembly's weights
  double SHW[ND], SWFE[ND], SWFT[ND], SHDC[ND], SCW[ND], SHWT[ND];
#pragma unroll
  for (int i = 0; i < ND; ++i) SHW[i] = SWFE[i] = SWFT[i] = SHDC[i] = SCW[i] = SHWT[i] = 0.0;
  double WDS_all = 0.0, HDP_all = 0.0, HDS_all = 0.0;   // terms of every species
  RX::each(m, [&](const auto& x, int r) {
    const D lnk = x.lnA() + x.b() * lnT - x.EaR() * invT;
    D M = cst<D>(1.0);
    if (x.type() != RX_ELEM) {
      M = Msum;
      for (int e = x.eff_begin(); e < x.eff_end(); ++e) M += x.eff_am1(m, e) * cget(x.eff_k(m, e));
    }
    const bool fo = (x.type() == RX_LINDEMANN || x.type() == RX_TROE);
    D kf, dlnkf, dkf_dM = cst<D>(0.0), phi = cst<D>(1.0);
    if (fo) {
      kf = falloff_s<D>(m, x, T, lnT, invT, M, sexp(m, lnk), dlnkf, dkf_dM, phi);
    } else {
      kf = sexp(m, lnk);
      dlnkf = (x.b() + x.EaR() * invT) * invT;
    }
    D kr = cst<D>(0.0), dlnKc = cst<D>(0.0);
    if (x.rev()) {
      D lnKc = x.dnu() * lnPRT;
      D dh = cst<D>(0.0);
      for (int q = 0; q < x.nf(); ++q) {
        lnKc += x.fod(q) * tget(HS::GV, HS::GD, x.fi(q));
        dh -= x.fod(q) * tget(HS::HV, HS::HD, x.fi(q));
      }
      for (int q = 0; q < x.nb(); ++q) {
        lnKc -= x.bod(q) * tget(HS::GV, HS::GD, x.bi(q));
        dh += x.bod(q) * tget(HS::HV, HS::HD, x.bi(q));
      }
      kr = fo ? kf * sexp(m, -lnKc) : sexp(m, lnk - lnKc);
      dlnKc = (dh - x.dnu()) * invT;
    }
    D cf[kMaxSide], cb[kMaxSide], pf[kMaxSide], pb[kMaxSide];
#pragma unroll
    for (int q = 0; q < kMaxSide; ++q) {
      cf[q] = (q < x.nf()) ? cget(x.fi(q)) : cst<D>(1.0);
      cb[q] = (q < x.nb()) ? cget(x.bi(q)) : cst<D>(1.0);
      pf[q] = (q < x.nf()) ? ipow_s(cf[q], x.fo(q)) : cst<D>(1.0);
      pb[q] = (q < x.nb()) ? ipow_s(cb[q], x.bo(q)) : cst<D>(1.0);
    }
    D Pf = pf[0], Pb = pb[0];
    if (x.nf() > 1) Pf = Pf * pf[1];
    if (x.nf() > 2) Pf = Pf * pf[2];
    if (x.nb() > 1) Pb = Pb * pb[1];
    if (x.nb() > 2) Pb = Pb * pb[2];
    const D q0 = kf * Pf - kr * Pb;
    const bool tb = (x.type() == RX_THREEBODY);
    const D mf = tb ? M : cst<D>(1.0);
    const D q = mf * q0;
    const D dqdT = mf * (kf * dlnkf * Pf - kr * (dlnkf - dlnKc) * Pb);
    double s1[ND];
#pragma unroll
    for (int i = 0; i < ND; ++i) s1[i] = 0.0;
    D s2 = cst<D>(0.0);
    for (int pp = 0; pp < x.np(); ++pp) {
      const int k = x.pi(pp);
#pragma unroll
      for (int i = 0; i < ND; ++i) s1[i] += w_at(i, k) * sp[k].W * x.pnu(pp);
      s2 += x.pnu(pp) * tget(HS::HV, HS::HD, k);
    }
    auto side = [&](int k, const D& gs) {
      double ws = 0.0, hs = 0.0;
#pragma unroll
      for (int i = 0; i < ND; ++i) {
        ws += s1[i] * gs.d[i];
        hs += wK[i] * fma(s2.v, gs.d[i], s2.d[i] * gs.v);
      }
      L[HS::WDS + k] += ws;
      L[HS::HDP + k] += s2.v * gs.v;
      L[HS::HDS + k] += hs;
    };
    // gradient of q w.r.t. each side's concentrations (added to the species at once) and grad q . c
    const D mkf = mf * kf, mkr = mf * kr;
    D gc = cst<D>(0.0);
#pragma unroll
    for (int s = 0; s < kMaxSide; ++s) {
      D of = cst<D>(1.0), ob = cst<D>(1.0);
#pragma unroll
      for (int t = 0; t < kMaxSide; ++t) {
        if (t != s && t < x.nf()) of = of * pf[t];
        if (t != s && t < x.nb()) ob = ob * pb[t];
      }
      if (s < x.nf()) {
        const D df = (x.fo(s) == 1) ? cst<D>(1.0) : (x.fo(s) == 2 ? 2.0 * cf[s] : 3.0 * (cf[s] * cf[s]));
        const D gf = mkf * df * of;
        gc += gf * cf[s];
        side(x.fi(s), gf);
      }
      if (s < x.nb()) {
        const D db = (x.bo(s) == 1) ? cst<D>(1.0) : (x.bo(s) == 2 ? 2.0 * cb[s] : 3.0 * (cb[s] * cb[s]));
        const D gb = -(mkr * db * ob);
        gc += gb * cb[s];
        side(x.bi(s), gb);
      }
    }
    D allc = cst<D>(0.0);
    if (tb) allc = q0;
    else if (fo) allc = (kf.v != 0.0) ? dkf_dM * (q0 / kf) : cst<D>(0.0);
    if (x.type() != RX_ELEM) gc += allc * M;
    const double invTv = invT.v;
    for (int pp = 0; pp < x.np(); ++pp) {
      const int k = x.pi(pp);
      const double nu = x.pnu(pp);
      const double hk = L[HS::HV + k], cpk = L[HS::PV + k];
      L[HS::WDP + k] += nu * q.v;
      L[HS::WTP + k] += nu * dqdT.v;
      L[HS::DCP + k] += nu * gc.v;
#pragma unroll
      for (int i = 0; i < ND; ++i) {
        const double wtk = w_at(i, k) * sp[k].W;
        const double dq = nu * q.d[i], dqt = nu * dqdT.d[i], dgc = nu * gc.d[i];
        SHW[i] += hk * dq;
        SCW[i] += cpk * dq;
        SWFE[i] += wtk * (dq - dgc);
        SWFT[i] += wtk * (dqt + (dq - dgc) * invTv);
        SHDC[i] += hk * dgc;
        SHWT[i] += hk * (dqt - dgc * invTv);
      }
    }
    if (x.type() != RX_ELEM) {
      const D a2 = s2 * allc;
      double a1s = 0.0, a2s = 0.0;
#pragma unroll
      for (int i = 0; i < ND; ++i) {
        a1s += s1[i] * allc.d[i];
        a2s += wK[i] * a2.d[i];
      }
      WDS_all += a1s;
      HDP_all += a2.v;
      HDS_all += a2s;
      for (int e = x.eff_begin(); e < x.eff_end(); ++e) {
        const int k = x.eff_k(m, e);
        const double am1 = x.eff_am1(m, e);
        L[HS::WDS + k] += a1s * am1;
        L[HS::HDP + k] += a2.v * am1;
        L[HS::HDS + k] += a2s * am1;
      }
    }
    // w_i^T df/dq_r = (s1_i - facT_i s2) / rho;  d q / d ln A = phi q;  d q / d E = -phi q / (R T)
    double dA = 0.0, dE = 0.0;
#pragma unroll
    for (int i = 0; i < ND; ++i) {
      const Dual sr = (s1[i] - facT[i] * view(s2, i)) * view(invrho, i);
      const Dual tA = sr * view(phi, i) * view(q, i);
      const Dual tE = -(tA / view(RT, i));
      dA += tA.d;
      dE += tE.d;
    }
    thA[r * stride] += dA;
    thE[r * stride] += dE;
  });
  // primal sums of the final assembly and their temperature-derivative parts
  double sum_hw = 0.0, HDc = 0.0, Cw = 0.0, HwT = 0.0, hdw = 0.0, hdc = 0.0, cdw = 0.0, hdwt = 0.0;
  double wfe[ND], wfT[ND];
#pragma unroll
  for (int i = 0; i < ND; ++i) wfe[i] = wfT[i] = 0.0;
  const double invTv = invT.v;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const double wd = L[HS::WDP + k], dc = L[HS::DCP + k], wt = L[HS::WTP + k];
    const double h = L[HS::HV + k], hd = L[HS::HD + k];
    sum_hw += h * wd;
    HDc += h * dc;
    Cw += L[HS::PV + k] * wd;
    HwT += h * (wt - dc * invTv);
    hdw += hd * wd;
    hdc += hd * dc;
    cdw += L[HS::PD + k] * wd;
    hdwt += hd * (wt - dc * invTv);
#pragma unroll
    for (int i = 0; i < ND; ++i) {
      const double wtk = w_at(i, k) * sp[k].W;
      wfe[i] += wtk * (wd - dc);
      wfT[i] += wtk * (wt + (wd - dc) * invTv);
    }
  }
  double Bbeta = 0.0, Acoef = 0.0, AwHDc = 0.0, Afcp = 0.0, AT = 0.0, AcpW = 0.0, gKs = 0.0;
  double coef_v = 0.0, wHDc_v = 0.0, fcp_v = 0.0, cpW_v = 0.0;
#pragma unroll
  for (int i = 0; i < ND; ++i) {
    const Dual Ti = view(T, i), invTi = view(invT, i), RTi = view(RT, i), invrhoi = view(invrho, i);
    const Dual cpm_Ji = view(cpm_J, i);
    const Dual sum_hwi = mk(sum_hw, Ti.d * hdw + SHW[i]);
    const Dual HDci = mk(HDc, Ti.d * hdc + SHDC[i]);
    const Dual Cwi = mk(Cw, Ti.d * cdw + SCW[i]);
    const Dual HwTi = mk(HwT, Ti.d * hdwt + SHWT[i] - HDc * invTi.d);
    const Dual wfei = mk(wfe[i], SWFE[i]);
    const Dual wfTi = mk(wfT[i], SWFT[i] + invTi.d * wfe[i]);
    const Dual fT = -(RTi * sum_hwi * invrhoi) / cpm_Ji;
    const Dual Wbar = 1.0 / view(sumYW, i);
    const Dual beta = Wbar * invrhoi * wfei;
    const Dual inv_cp = 1.0 / cpm_Ji;
    const Dual coef = -(RTi * inv_cp);
    const Dual wHDc = Wbar * invrhoi * HDci;
    const Dual fcp = fT * inv_cp;
    const Dual cpW = cpm_Ji * Wbar;
    Bbeta += beta.d;
    Acoef += wK[i] * coef.d;
    AwHDc += wK[i] * wHDc.d;
    Afcp += wK[i] * fcp.d;
    AT += wK[i] * Ti.d;
    AcpW += wK[i] * cpW.d;
    coef_v = coef.v;
    wHDc_v = wHDc.v;
    fcp_v = fcp.v;
    cpW_v = cpW.v;
    const Dual JTT = -((kRu * Cwi + RTi * HwTi) * invrhoi * inv_cp) + fT * invTi - fT * (kRu * view(dcpm, i)) * inv_cp;
    const Dual gT = invrhoi * wfTi + wK[i] * JTT;
    gKs += gT.d;
  }
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const double hdv = L[HS::HDP + k] + HDP_all;
    const double gi = Acoef * (hdv - wHDc_v) + coef_v * (L[HS::HDS + k] + HDS_all - AwHDc) -
                      Afcp * (kRu * L[HS::PV + k] - cpW_v) - fcp_v * (kRu * L[HS::PD + k] * AT - AcpW);
    g[k] += sp[k].Winv * (L[HS::WDS + k] + WDS_all + Bbeta + gi);
  }
  g[K] += gKs;
}

// ---------------------------------------------------------------------------
// kernel 1: record the accepted steps of every cell's forward integration
// ---------------------------------------------------------------------------
struct AdjArgs {
  const unsigned char* mech;
  const unsigned char* plan;   // gather plan of the CTA-per-cell kernels (null for thread per cell)
  int mech_bytes;
  int K, R;
  long long n;
  const double* p;
  const double* T0;
  const double* Y0;
  long long ldY;
  double dt;
  rde_chem_options opt;
  const int* n_steps;          // [n] accepted steps of the forward pass
  long long total_steps;       // records the pool (and stages) hold
  const long long* order;      // [n] cells by accepted steps, most first (null: index order)
  long long* offsets;          // [n + 1] exclusive scan of n_steps
  double* pool;                // [sum n_steps][N + 1]: y_n then h_n
  double* stages;              // null, or [sum n_steps][N N + 4 N + 1]: the step's LU factors
                               // (1/U_kk on the diagonal), pivot word, u_1 .. u_4
  int* rec;                    // [n] steps recorded (or -status on failure)
  const double* gT;            // [n]
  const double* gY;            // [K][ldY]
  double* gT0;                 // [n]
  double* gY0;                 // [K][ldY]
  double* lane_scratch;        // [(8 N + 2 R) x lanes]
  double* rows;                // [2 R][n] per-cell parameter cotangents
  unsigned long long* queue;   // [2] work-queue counters (record, reverse)
  int* status;                 // optional [n]
  int num_sms;
  // self-checkpointing mode (n_steps == null: the step counts are not known in advance)
  int ckpt_S;                  // checkpoint entries per cell (a power of two), 0 otherwise
  int seg_max;                 // largest checkpoint stride the options allow (power of two)
  double* ckpt;                // [n][ckpt_S][N + 3]: y_n, t_n, the proposed step size at t_n, h_n
  double* seg;                 // [seg_max][N + 1][lanes]: the replayed y_n, h_n of one segment
  double* replay;              // [N + 6][lanes]: replay state y, t, h, rejected flag, count, target, attempts
};

// The adjoint's copy of the forward attempt, compiled once (not inlined) so that the
// record pass and the reverse sweep's segment replays run the very same instructions:
// a replayed segment then retraces the recorded steps bit for bit.
template <int K, class RX>
__device__ __noinline__ bool adj_attempt(const MechView m, const Lane L, double invp, const double* y, double h,
                                         const Opts o, double* yn, double* err, bool* finite,
                                         unsigned long long* swaps, double* U) {
  constexpr int N = K + 1;
  double yv[N], ynv[N], Uv[4][N];
#pragma unroll
  for (int i = 0; i < N; ++i) yv[i] = y[i];
  const bool ok = rosenbrock_attempt<K, RhsOf<RX>, kMethodRodas3, true>(m, L, invp, yv, h, o, ynv, *err, *finite,
                                                                        *swaps, Uv);
#pragma unroll
  for (int i = 0; i < N; ++i) {
    yn[i] = ynv[i];
    U[i] = Uv[0][i];
    U[N + i] = Uv[1][i];
    U[2 * N + i] = Uv[2][i];
    U[3 * N + i] = Uv[3][i];
  }
  return ok;
}

// Stride of a cell's checkpoints in self-checkpointing mode: the smallest power of two
// s with nrec <= S s (the record pass thins its S entries to every other one whenever
// they are full, so entry e holds step e s).
__host__ __device__ __forceinline__ int ckpt_stride(int nrec, int S) {
  int s = 1;
  while ((long long)S * s < (long long)nrec) s <<= 1;
  return s;
}

template <int K, class RX>
__device__ __forceinline__ void record_body(const AdjArgs& a) {
  using S = Slots<K>;
  constexpr int N = K + 1;
  extern __shared__ __align__(16) unsigned char smem[];
  {
    const int4* src = reinterpret_cast<const int4*>(a.mech);
    int4* dst = reinterpret_cast<int4*>(smem);
    for (int i = threadIdx.x; i < a.mech_bytes / 16; i += blockDim.x) dst[i] = src[i];
  }
  __syncthreads();
  const MechView m = mech_view(smem);
  const Lane L{reinterpret_cast<double*>(smem + a.mech_bytes) + threadIdx.x};
  const int lane = threadIdx.x & 31;
  const Opts o{a.opt.rtol, a.opt.atol, a.opt.h_min, a.opt.facmax, a.opt.facmin, a.opt.safety, a.opt.max_substeps, 0};
  const double dt = a.dt;
  bool active = false, exhausted = false;
  long long cell = 0, off = 0;
  int cap = 0, nrec = 0, attempts = 0;
  double y[N];
  double invp = 0.0, t = 0.0, h = 0.0;
  bool reject_prev = false;
  const bool self = a.ckpt_S > 0;
  int stride = 1;      // self mode: current checkpoint stride
  double hp0 = 0.0;    // self mode: the step size proposed for the next step (before any rejection)
  for (;;) {
    bool need = !active && !exhausted;
    while (__any_sync(kFullA, need)) {
      const unsigned mask = __ballot_sync(kFullA, need);
      const int leader = __ffs(mask) - 1;
      unsigned long long base = 0;
      if (lane == leader) base = atomicAdd(a.queue, (unsigned long long)__popc(mask));
      base = __shfl_sync(kFullA, base, leader);
      if (need) {
        const long long q = (long long)(base + __popc(mask & ((1u << lane) - 1u)));
        // queue position q holds the q-th cell of the cost order (most accepted steps first)
        const long long g = (q < a.n && a.order) ? a.order[q] : q;
        if (q >= a.n) {
          exhausted = true;
          need = false;
        } else if (g < 0 || g >= a.n) {
          // an order entry outside [0, n): nothing to do for this position
        } else {
          cell = g;
          const double p = a.p[g];
          bool good = isfinite(p) && p > 0.0;
#pragma unroll
          for (int k = 0; k < K; ++k) {
            y[k] = a.Y0[k * a.ldY + g];
            good = good && isfinite(y[k]);
          }
          y[K] = a.T0[g];
          good = good && isfinite(y[K]) && y[K] > 0.0;
          invp = 1.0 / p;
          t = 0.0;
          h = dt;
          nrec = attempts = 0;
          reject_prev = false;
          stride = 1;
          hp0 = h;
          bool room = true;
          if (!self) {
            off = a.offsets[g];
            cap = (int)(a.offsets[g + 1] - off);
            // the caller's total_steps is below the sum of n_steps: no room for this cell
            room = a.offsets[g + 1] <= a.total_steps;
          }
          if (!room) {
            a.rec[g] = -RDE_CELL_ADJ_MISMATCH;
          } else if (good) {
            active = true;
            need = false;
          } else {
            a.rec[g] = -RDE_CELL_BAD_STATE;
          }
        }
      }
    }
    if (!__any_sync(kFullA, active)) break;
    if (active) {
      int fail = 0;
      if (attempts >= o.max_substeps) {
        fail = RDE_CELL_MAX_SUBSTEPS;
      } else {
        ++attempts;
        h = fmin(h, dt - t);
        // the forward kernel's attempt, in the one compiled copy the replays share
        double yn[N], err, U[4][N];
        bool finite;
        unsigned long long swaps;
        if (!adj_attempt<K, RX>(m, L, invp, y, h, o, yn, &err, &finite, &swaps, &U[0][0])) {
          fail = RDE_CELL_LU_SINGULAR;
        } else if (finite && err <= 1.0) {
          if (self) {
            // checkpoint of this step at every stride-th step; when the S entries are full,
            // keep every other one and double the stride
            if ((nrec & (stride - 1)) == 0) {
              double* base = a.ckpt + cell * (long long)a.ckpt_S * (N + 3);
              int e = nrec / stride;
              if (e == a.ckpt_S) {
#pragma unroll 1
                for (int q = 1; q < a.ckpt_S / 2; ++q) {
#pragma unroll
                  for (int f = 0; f < N + 3; ++f) base[q * (N + 3) + f] = base[2 * q * (N + 3) + f];
                }
                stride <<= 1;
                e = a.ckpt_S / 2;
              }
              double* en = base + (long long)e * (N + 3);
#pragma unroll
              for (int i = 0; i < N; ++i) en[i] = y[i];
              en[N] = t;
              en[N + 1] = hp0;
              en[N + 2] = h;
            }
          } else if (nrec < cap) {
            double* rec = a.pool + (off + nrec) * (N + 1);
#pragma unroll
            for (int i = 0; i < N; ++i) rec[i] = y[i];
            rec[N] = h;
            if (a.stages) {
              // stage checkpoint: the LU factors as lu_factor leaves them (1/U_kk on the
              // diagonal), the interchanges as 4-bit fields of one word, the four stages
              double* cp = a.stages + (off + nrec) * (long long)(N * N + 4 * N + 1);
#pragma unroll 1
              for (int r = 0; r < N; ++r) {
#pragma unroll 2
                for (int c = 0; c < N; ++c) cp[r * N + c] = L[S::MX + r * N + c];
              }
              cp[N * N] = __longlong_as_double((long long)swaps);
#pragma unroll
              for (int i = 0; i < N; ++i) {
                cp[N * N + 1 + i] = U[0][i];
                cp[N * N + 1 + N + i] = U[1][i];
                cp[N * N + 1 + 2 * N + i] = U[2][i];
                cp[N * N + 1 + 3 * N + i] = U[3][i];
              }
            }
          }
          ++nrec;
#pragma unroll
          for (int i = 0; i < N; ++i) y[i] = yn[i];
          t += h;
          h *= step_factor<kMethodRodas3>(err, finite, true, reject_prev, o);
          hp0 = h;
          reject_prev = false;
          if (dt - t <= 1e-14 * dt) {
            a.rec[cell] = (self || nrec == cap) ? nrec : -RDE_CELL_ADJ_MISMATCH;
            active = false;
          }
        } else {
          h *= step_factor<kMethodRodas3>(err, finite, false, reject_prev, o);
          reject_prev = true;
          if (h < o.hmin) fail = RDE_CELL_H_UNDERFLOW;
        }
      }
      if (fail) {
        a.rec[cell] = -fail;
        active = false;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// kernel 2: reverse sweep
// ---------------------------------------------------------------------------
template <int K, class RX, int ND = 1, bool SELF = false>
__device__ __forceinline__ void reverse_body(const AdjArgs& a) {
  static_assert(ND == 1 || ND == 2 || ND == 4, "the four stages split into evaluations of ND directions");
  using S = AdjSlots<K>;
  constexpr int N = K + 1;
  extern __shared__ __align__(16) unsigned char smem[];
  {
    const int4* src = reinterpret_cast<const int4*>(a.mech);
    int4* dst = reinterpret_cast<int4*>(smem);
    for (int i = threadIdx.x; i < a.mech_bytes / 16; i += blockDim.x) dst[i] = src[i];
  }
  __syncthreads();
  const MechView m = mech_view(smem);
  const Lane L{reinterpret_cast<double*>(smem + a.mech_bytes) + threadIdx.x};
  const int lane = threadIdx.x & 31;
  const long long nl = (long long)gridDim.x * blockDim.x;
  const long long me = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double* U = a.lane_scratch + me;                  // U[(i*N + e) * nl]
  double* W = a.lane_scratch + 4 * N * nl + me;     // W[(i*N + e) * nl]
  double* thA = a.lane_scratch + 8 * N * nl + me;   // thA[r * nl]
  double* thE = thA + (long long)a.R * nl;
  bool active = false, exhausted = false;
  long long cell = 0, off = 0;
  int s = 0;
  double lam[N];
  double invp = 0.0;
  // self-checkpointing mode: the cell's checkpoint stride, whether the lane is replaying
  // a segment, the first step the segment buffer holds and the cell's step count
  int cs = 1, seg0 = 0, ncell = 0;
  bool replaying = false;
  double* Rp = a.replay + me;                       // Rp[f * nl], f < N + 6
  double* Sg = a.seg + me;                          // Sg[(q * (N + 1) + f) * nl]
  const double* Ck = nullptr;                       // the cell's checkpoints
  // start replaying segment j (steps j cs .. ) from its checkpoint
  auto begin_replay = [&](int j) {
    const double* en = Ck + (long long)j * (N + 3);
#pragma unroll
    for (int i = 0; i < N; ++i) Rp[i * nl] = en[i];
    Rp[N * nl] = en[N];            // t
    Rp[(N + 1) * nl] = en[N + 1];  // proposed step size
    Rp[(N + 2) * nl] = 0.0;        // previous attempt rejected
    Rp[(N + 3) * nl] = 0.0;        // steps replayed
    Rp[(N + 4) * nl] = (double)min(cs, ncell - j * cs);
    Rp[(N + 5) * nl] = 0.0;        // attempts
    seg0 = j * cs;
    replaying = true;
  };
  // the cell's gradients are zero and its status `st` (failed forward or replay)
  auto fail_cell = [&](int st) {
    if (a.status) a.status[cell] = st;
#pragma unroll
    for (int k = 0; k < K; ++k) a.gY0[k * a.ldY + cell] = 0.0;
    a.gT0[cell] = 0.0;
    for (int j = 0; j < 2 * a.R; ++j) a.rows[(long long)j * a.n + cell] = 0.0;
    active = false;
  };
  for (;;) {
    bool need = !active && !exhausted;
    while (__any_sync(kFullA, need)) {
      const unsigned mask = __ballot_sync(kFullA, need);
      const int leader = __ffs(mask) - 1;
      unsigned long long base = 0;
      if (lane == leader) base = atomicAdd(a.queue + 1, (unsigned long long)__popc(mask));
      base = __shfl_sync(kFullA, base, leader);
      if (need) {
        const long long q = (long long)(base + __popc(mask & ((1u << lane) - 1u)));
        // queue position q holds the q-th cell of the cost order (most accepted steps first)
        const long long g = (q < a.n && a.order) ? a.order[q] : q;
        if (q >= a.n) {
          exhausted = true;
          need = false;
        } else if (g < 0 || g >= a.n) {
          // an order entry outside [0, n): nothing to do for this position
        } else {
          cell = g;
          const int nrec = a.rec[g];
          if (a.status) a.status[g] = nrec > 0 ? RDE_CELL_OK : -nrec;
          for (int j = 0; j < 2 * a.R; ++j) thA[(long long)j * nl] = 0.0;
          if (nrec <= 0) {
            // failed or inconsistent forward: no gradient
#pragma unroll
            for (int k = 0; k < K; ++k) a.gY0[k * a.ldY + g] = 0.0;
            a.gT0[g] = 0.0;
            for (int j = 0; j < 2 * a.R; ++j) a.rows[(long long)j * a.n + g] = 0.0;
          } else {
            s = nrec - 1;
#pragma unroll
            for (int k = 0; k < K; ++k) lam[k] = a.gY[k * a.ldY + g];
            lam[K] = a.gT[g];
            invp = 1.0 / a.p[g];
            active = true;
            need = false;
            if constexpr (SELF) {
              ncell = nrec;
              cs = ckpt_stride(nrec, a.ckpt_S);
              Ck = a.ckpt + g * (long long)a.ckpt_S * (N + 3);
              replaying = false;
              if (cs > 1) begin_replay(s / cs);
            } else {
              off = a.offsets[g];
            }
          }
        }
      }
    }
    if (!__any_sync(kFullA, active)) break;
    if constexpr (SELF) {
      if (active && replaying) {
        // ---- one attempt of the segment's replay (the record pass's arithmetic) ----
        double ry[N], yn[N], err, unused[4][N];
#pragma unroll
        for (int i = 0; i < N; ++i) ry[i] = Rp[i * nl];
        const double rt = Rp[N * nl];
        const double hatt = fmin(Rp[(N + 1) * nl], a.dt - rt);
        const bool rrej = Rp[(N + 2) * nl] != 0.0;
        int rcnt = (int)Rp[(N + 3) * nl];
        const int rtarget = (int)Rp[(N + 4) * nl];
        const double ratt = Rp[(N + 5) * nl] + 1.0;
        Rp[(N + 5) * nl] = ratt;
        bool finite;
        unsigned long long swaps;
        const Opts o{a.opt.rtol, a.opt.atol, a.opt.h_min, a.opt.facmax, a.opt.facmin, a.opt.safety,
                     a.opt.max_substeps, 0};
        if (ratt > (double)o.max_substeps ||
            !adj_attempt<K, RX>(m, L, invp, ry, hatt, o, yn, &err, &finite, &swaps, &unused[0][0])) {
          fail_cell(RDE_CELL_ADJ_MISMATCH);
        } else if (finite && err <= 1.0) {
#pragma unroll
          for (int i = 0; i < N; ++i) Sg[(rcnt * (N + 1) + i) * nl] = ry[i];
          Sg[(rcnt * (N + 1) + N) * nl] = hatt;
          ++rcnt;
#pragma unroll
          for (int i = 0; i < N; ++i) Rp[i * nl] = yn[i];
          Rp[N * nl] = rt + hatt;
          Rp[(N + 1) * nl] = hatt * step_factor<kMethodRodas3>(err, finite, true, rrej, o);
          Rp[(N + 2) * nl] = 0.0;
          Rp[(N + 3) * nl] = (double)rcnt;
          if (rcnt == rtarget) {
            replaying = false;
            // the replayed segment must end on the next checkpoint, bit for bit
            const int jn = (seg0 + rcnt) / cs;
            if (seg0 + rcnt < ncell) {
              const double* en = Ck + (long long)jn * (N + 3);
              bool same = en[N] == rt + hatt;
#pragma unroll
              for (int i = 0; i < N; ++i) same = same && (__double_as_longlong(en[i]) == __double_as_longlong(yn[i]));
              if (!same) fail_cell(RDE_CELL_ADJ_MISMATCH);
            }
          }
        } else {
          const double hn = hatt * step_factor<kMethodRodas3>(err, finite, false, rrej, o);
          Rp[(N + 1) * nl] = hn;
          Rp[(N + 2) * nl] = 1.0;
          if (hn < o.hmin) fail_cell(RDE_CELL_ADJ_MISMATCH);
        }
        continue;
      }
    }
    if (active) {
      double y[N];
      const double* rec;
      int rstride = N + 1;
      if constexpr (SELF) {
        if (cs == 1) {
          rec = Ck + (long long)s * (N + 3);
          rstride = 1;
        } else {
          rec = Sg + (long long)(s - seg0) * (N + 1) * nl;
          rstride = 0;
        }
      } else {
        rec = a.pool + (off + s) * (N + 1);
        rstride = 1;
      }
      double h;
      if (rstride == 0) {
#pragma unroll
        for (int i = 0; i < N; ++i) y[i] = rec[i * nl];
        h = rec[N * nl];
      } else {
#pragma unroll
        for (int i = 0; i < N; ++i) y[i] = rec[i];
        h = (SELF) ? rec[N + 2] : rec[N];
      }
      const double invh = 1.0 / h;
      unsigned long long piv;
      if (a.stages) {
        // ---- the stages of this step from its checkpoint ----
        const double* cp = a.stages + (off + s) * (long long)(N * N + 4 * N + 1);
#pragma unroll 4
        for (int e = 0; e < N * N; ++e) L[S::MX + e] = cp[e];
        piv = (unsigned long long)__double_as_longlong(cp[N * N]);
#pragma unroll
        for (int i = 0; i < 4 * N; ++i) U[i * nl] = cp[N * N + 1 + i];
      } else {
        // ---- recompute the stages of this step ----
#pragma unroll
        for (int i = 0; i < N; ++i) L[S::ARG + i] = y[i];
        const MixState ms = RhsOf<RX>::template eval<K, true, S>(m, L, invp);
        double f0[N];
#pragma unroll
        for (int i = 0; i < N; ++i) f0[i] = L[S::VEC + i];
        assemble_matrix<K, S>(m, L, y[K], ms, 1.0 / (kGamma * h), invp);
        lu_factor_r<K>(L, piv);
        {
          double u1[N], u2[N], u3[N];
          lu_solve_r<K>(L, piv);
#pragma unroll
          for (int i = 0; i < N; ++i) u1[i] = L[S::VEC + i];
#pragma unroll
          for (int i = 0; i < N; ++i) L[S::VEC + i] = f0[i] + (kC21 * invh) * u1[i];
          lu_solve_r<K>(L, piv);
#pragma unroll
          for (int i = 0; i < N; ++i) {
            u2[i] = L[S::VEC + i];
            L[S::ARG + i] = y[i] + 2.0 * u1[i];
          }
          RhsOf<RX>::template eval<K, false, S>(m, L, invp);
#pragma unroll
          for (int i = 0; i < N; ++i) L[S::VEC + i] += invh * (u1[i] - u2[i]);
          lu_solve_r<K>(L, piv);
#pragma unroll
          for (int i = 0; i < N; ++i) {
            u3[i] = L[S::VEC + i];
            L[S::ARG + i] = y[i] + 2.0 * u1[i] + u3[i];
          }
          RhsOf<RX>::template eval<K, false, S>(m, L, invp);
#pragma unroll
          for (int i = 0; i < N; ++i) L[S::VEC + i] += invh * (u1[i] - u2[i] + kC43 * u3[i]);
          lu_solve_r<K>(L, piv);
#pragma unroll
          for (int i = 0; i < N; ++i) {
            U[(0 * N + i) * nl] = u1[i];
            U[(1 * N + i) * nl] = u2[i];
            U[(2 * N + i) * nl] = u3[i];
            U[(3 * N + i) * nl] = L[S::VEC + i];
          }
        }
      }
      // ---- adjoint of the stages: ybar = lam; ubar4 = lam, ubar3 = lam, ubar2 = 0, ubar1 = 2 lam ----
      double yb[N], ub1[N], ub2[N], ub3[N], g[N], arg[N], w[N];
#pragma unroll
      for (int i = 0; i < N; ++i) {
        yb[i] = lam[i];
        ub1[i] = 2.0 * lam[i];
        ub2[i] = 0.0;
        ub3[i] = lam[i];
        L[S::VEC + i] = lam[i];
      }
      // stage 4: r4 = f(y + 2 u1 + u3) + (u1 - u2 + c43 u3)/h
      lu_solve_t<K>(L, piv);
#pragma unroll
      for (int i = 0; i < N; ++i) {
        w[i] = L[S::VEC + i];
        W[(3 * N + i) * nl] = w[i];
        arg[i] = y[i] + 2.0 * U[(0 * N + i) * nl] + U[(2 * N + i) * nl];
      }
      jtw<K, double, RX>(m, L, S::C, invp, arg, w, g, thA, thE, nl);
#pragma unroll
      for (int i = 0; i < N; ++i) {
        yb[i] += g[i];
        ub1[i] += 2.0 * g[i] + invh * w[i];
        ub2[i] -= invh * w[i];
        ub3[i] += g[i] + (kC43 * invh) * w[i];
        L[S::VEC + i] = ub3[i];
      }
      // stage 3: r3 = f(y + 2 u1) + (u1 - u2)/h
      lu_solve_t<K>(L, piv);
#pragma unroll
      for (int i = 0; i < N; ++i) {
        w[i] = L[S::VEC + i];
        W[(2 * N + i) * nl] = w[i];
        arg[i] = y[i] + 2.0 * U[(0 * N + i) * nl];
      }
      jtw<K, double, RX>(m, L, S::C, invp, arg, w, g, thA, thE, nl);
#pragma unroll
      for (int i = 0; i < N; ++i) {
        yb[i] += g[i];
        ub1[i] += 2.0 * g[i] + invh * w[i];
        ub2[i] -= invh * w[i];
        L[S::VEC + i] = ub2[i];
      }
      // stage 2: r2 = f(y) + (c21/h) u1
      lu_solve_t<K>(L, piv);
#pragma unroll
      for (int i = 0; i < N; ++i) {
        w[i] = L[S::VEC + i];
        W[(1 * N + i) * nl] = w[i];
        ub1[i] += (kC21 * invh) * w[i];
        L[S::VEC + i] = ub1[i];
      }
      // stage 1: r1 = f(y)
      lu_solve_t<K>(L, piv);
#pragma unroll
      for (int i = 0; i < N; ++i) {
        const double w1 = L[S::VEC + i];
        W[(0 * N + i) * nl] = w1;
        w[i] = w1 + W[(1 * N + i) * nl];   // f(y) enters stages 1 and 2
      }
      jtw<K, double, RX>(m, L, S::C, invp, y, w, g, thA, thE, nl);
#pragma unroll
      for (int i = 0; i < N; ++i) yb[i] += g[i];
      // ---- M = I/(gamma h) - J(y): terms grad (w_i^T J(y) u_i) ----
      if constexpr (ND > 1) {
        // ND stages per evaluation, sharing its primal part
#pragma unroll 1
        for (int st = 0; st < 4; st += ND) hvp_sum<K, ND, RX>(m, L, invp, y, U, W, st, nl, yb, thA, thE, nl);
      } else {
        // one dual-number evaluation per stage
#pragma unroll 1
      for (int st = 0; st < 4; ++st) {
        Dual yd[N];
#pragma unroll
        for (int i = 0; i < N; ++i) {
          yd[i] = mk(y[i], U[(st * N + i) * nl]);
          w[i] = W[(st * N + i) * nl];
        }
        jtw<K, Dual, RX>(m, L, 0, invp, yd, w, g, thA, thE, nl);
#pragma unroll
        for (int i = 0; i < N; ++i) yb[i] += g[i];
      }
      }
#pragma unroll
      for (int i = 0; i < N; ++i) lam[i] = yb[i];
      if (--s < 0) {
#pragma unroll
        for (int k = 0; k < K; ++k) a.gY0[k * a.ldY + cell] = lam[k];
        a.gT0[cell] = lam[K];
        for (int j = 0; j < 2 * a.R; ++j) a.rows[(long long)j * a.n + cell] = thA[(long long)j * nl];
        active = false;
      } else if constexpr (SELF) {
        if (cs > 1 && s < seg0) begin_replay(s / cs);
      }
    }
  }
}

}  // namespace rde
