// Device arithmetic of the per-cell chemistry step (sm_103a, FP64).
//
// One lane integrates one cell.  All lanes of a warp run the same substep code
// on different cells, so every mechanism-table read is a broadcast and the FP64
// pipe sees full warps.  On GB300 the FP64 pipe retires about two lane-operations
// per SM clock (1.20 TFLOP/s measured for the GPU), a warp instruction costs the
// same whether 1 or 32 lanes are active, and a dependent FP64 operation waits
// about one pipe slot (~64 cycles).  Integer, select and shared-memory work is
// therefore nearly free, while instruction-cache misses and long memory latency
// are not: the per-lane matrix and species arrays live in shared memory as
// per-thread slices ("lane slots": element e of thread t at [e][t], so a warp's
// access to one element is a conflict-free 256-byte row), loops are kept compact,
// and nothing spills to local memory.
//
// Model (Appendix A, Eqs. 20-21, closed adiabatic constant-pressure reactor):
//   c_k = rho Y_k / W_k,  rho = p / (R_u T sum_k Y_k / W_k)
//   k_f = exp(ln A + b ln T - E/(R_u T));  ln K_c = -sum_k nu_k G_k/RT + (sum nu) ln(P_std / (R_u T))
//   k_r = exp(ln k_f - ln K_c)  (reversible reactions)
//   q   = k_f prod c^nu' - k_r prod c^nu''  (times [M] for plain third-body reactions;
//         Lindemann / Troe blending k = k_inf Pr/(1+Pr) F, Pr = k_0 [M] / k_inf)
//   dY_k/dt = W_k omega_k / rho,  dT/dt = -R_u T sum_k (H/RT)_k omega_k / (rho c_p)
#pragma once
#if !defined(__CUDACC_RTC__)  /* run-time compilation: types from the preamble */
#include <cuda_runtime.h>
#include <stdint.h>
#endif

#include "fastmath.cuh"
#include "mech_layout.h"

namespace rde {

constexpr double kRu = 8.31446261815324;             // J/(mol K)
constexpr double kLnPstdOverRu = 9.408091968943316;  // ln(101325 Pa / R_u)
constexpr double kLn10 = 2.302585092994046;
constexpr double kInvLn10 = 0.43429448190325182;

// RODAS3 (Sandu et al. 1997) in the transformed form
//   (I/(h gamma) - J) u_i = f(y + sum_j a_ij u_j) + sum_j (c_ij / h) u_j
// with gamma = 1/2; a31 = 2, a41 = 2, a43 = 1 (others 0); c21 = 4, c31 = 1,
// c32 = -1, c41 = 1, c42 = -1, c43 = -8/3; y_new = y + 2 u1 + u3 + u4; error = u4.
constexpr double kGamma = 0.5;
constexpr double kC21 = 4.0, kC43 = -8.0 / 3.0;

// ROS2, the two-stage L-stable Rosenbrock method of order 2 with the embedded
// order-1 solution y + k1: classical gamma = 1 - 1/sqrt(2), alpha21 = 1,
// gamma21 = -2 gamma (beta21 = 1 - 2 gamma), b = (1/2, 1/2).  Transformed form:
// a21 = 1/gamma, c21 = (beta21 - alpha21)/gamma^2 = -2/gamma, m = b Gamma^-1 and
// the error weights e = (b - (1, 0)) Gamma^-1, which are equal for both stages.
constexpr int kMethodRodas3 = 0, kMethodRos2 = 1;
// Method 2: linearly implicit Euler extrapolation of fixed order 3 (the SEULEX
// family): for n_j = 1, 2, 3 substeps of h_j = H / n_j,
//   (I/h_j - J)(y_{i+1} - y_i) = f(y_i),  T_j1 = y_{n_j},  J = J(y) for all of them,
// Aitken-Neville for an error expansion in powers of h:
//   T21 = T2 + (T2 - T1),  T31 = T3 + 2 (T3 - T2),  T32 = T31 + (T31 - T21) / 2;
// y_new = T32 (order 3), error estimate T32 - T31 (order 2, exponent 1/3).
constexpr int kMethodExtrap = 2;
constexpr double kR2Gamma = 0.29289321881345248;
constexpr double kR2A21 = 3.4142135623730949, kR2C21 = -6.8284271247461898;
constexpr double kR2M1 = 5.1213203435596428, kR2M2 = 1.7071067811865475;
constexpr double kR2E = 1.7071067811865475;

constexpr int kLaneThreads = 128;   // threads per CTA: the stride of a lane slot

struct Opts {
  double rtol, atol, hmin, facmax, facmin, safety;
  int max_substeps;
  int method;   // kMethodRodas3 or kMethodRos2
};

// A thread's slice of the shared lane slots: element e at base[e * kLaneThreads].
// Every slot lives in shared memory; sm(e) is the same slot (the accessor the
// matrix code uses, since its indices may be run-time values).
struct Lane {
  static constexpr bool kRegs = false;   // no register-resident slots
  static constexpr int kUnroll = 3;      // unroll of the loops over species
  static constexpr int kUnrollOuter = 1; // unroll of the outer loops of the Jacobian assembly
  double* base;
  __device__ __forceinline__ double& operator[](int e) const { return base[e * kLaneThreads]; }
  __device__ __forceinline__ double& sm(int e) const { return base[e * kLaneThreads]; }
};

// Slot map of one lane for K species (N = K + 1 unknowns).
template <int K>
struct Slots {
  static constexpr int N = K + 1;
  static constexpr int MX = 0;              // N x N: D, then J, then I/(h gamma) - J, then its LU (1/U_kk on the diagonal)
  static constexpr int C = MX + N * N;      // concentrations
  static constexpr int G = C + K;           // G/RT  (reused as D c during assembly)
  static constexpr int HRT = G + K;         // H/RT
  static constexpr int CPR = HRT + K;       // Cp/R
  static constexpr int WDOT = CPR + K;      // net molar production
  static constexpr int WT = WDOT + K;       // d wdot / dT at fixed c
  static constexpr int ARG = WT + K;        // state argument of f (N)
  static constexpr int VEC = ARG + N;       // f output / right-hand side of a solve (N)
  static constexpr int TOTAL = VEC + N;
  static constexpr size_t bytes(int threads) { return sizeof(double) * TOTAL * threads; }
};

// Lane slots of the wide (two warps per SM sub-partition) kernels: only the N x N
// matrix stays in shared memory (element e of thread t at base[e * STRIDE]); the
// species and vector slots of Slots<K> are a per-thread array that the compiler keeps
// in registers, which needs every access to them to have a compile-time index (the
// reaction sequence and the loops over species are fully unrolled).  The matrix is
// reached through sm(), whose indices may be run-time values (pivot rows).
template <int K, int STRIDE>
struct RegLane {
  static constexpr bool kRegs = true;
  static constexpr int kUnroll = 64;        // >= K: full unroll
  static constexpr int kUnrollOuter = 64;
  static constexpr int NN = (K + 1) * (K + 1);
  static_assert(Slots<K>::MX == 0, "the matrix leads the slot map");
  double* base;
  mutable double r[Slots<K>::TOTAL - NN];
  __device__ __forceinline__ double& operator[](int e) const { return e < NN ? base[e * STRIDE] : r[e - NN]; }
  __device__ __forceinline__ double& sm(int e) const { return base[e * STRIDE]; }
};

// Bit pattern helpers: for non-negative finite doubles the integer order of the bit
// patterns is the numeric order, so magnitude comparisons and maxima can be taken on
// the integer pipe (the FP64 pipe is the scarce one on this GPU).
constexpr unsigned long long kAbsMask = 0x7fffffffffffffffull;
constexpr unsigned long long kExpMask = 0x7ff0000000000000ull;

__device__ __forceinline__ unsigned long long abs_bits(double x) {
  return (unsigned long long)__double_as_longlong(x) & kAbsMask;
}
__device__ __forceinline__ bool finite_bits(double x) {
  return ((unsigned long long)__double_as_longlong(x) & kExpMask) != kExpMask;
}

__device__ __forceinline__ double ipow(double c, int e) {
  double r = c;
  if (e >= 2) r *= c;
  if (e >= 3) r *= c;
  return r;
}

// Reaction descriptors.  The reaction term below reads a reaction through a
// descriptor: RxView reads the packed record of the mechanism image (the generic
// kernels loop over reactions), while a mechanism-specialised kernel passes one
// generated descriptor type per reaction whose structural members (type, species,
// orders, coefficients, falloff constants, efficiencies) are compile-time constants
// and whose ln A and E/R are still read from the image (so parameter updates need
// no recompilation).  Both run the same arithmetic in the same order.
struct RxView {
  const RxnPacked& x;
  __device__ __forceinline__ int type() const { return x.type; }
  __device__ __forceinline__ int rev() const { return x.rev; }
  __device__ __forceinline__ int nf() const { return x.nf; }
  __device__ __forceinline__ int nb() const { return x.nb; }
  __device__ __forceinline__ int np() const { return x.np; }
  __device__ __forceinline__ int fi(int q) const { return x.fi[q]; }
  __device__ __forceinline__ int fo(int q) const { return x.fo[q]; }
  __device__ __forceinline__ int bi(int q) const { return x.bi[q]; }
  __device__ __forceinline__ int bo(int q) const { return x.bo[q]; }
  __device__ __forceinline__ int pi(int q) const { return x.pi[q]; }
  __device__ __forceinline__ double fod(int q) const { return x.fod[q]; }
  __device__ __forceinline__ double bod(int q) const { return x.bod[q]; }
  __device__ __forceinline__ double pnu(int q) const { return x.pnu[q]; }
  __device__ __forceinline__ double lnA() const { return x.lnA; }
  __device__ __forceinline__ double EaR() const { return x.EaR; }
  __device__ __forceinline__ double b() const { return x.b; }
  __device__ __forceinline__ double dnu() const { return x.dnu; }
  __device__ __forceinline__ double lnA0() const { return x.lnA0; }
  __device__ __forceinline__ double b0() const { return x.b0; }
  __device__ __forceinline__ double EaR0() const { return x.EaR0; }
  __device__ __forceinline__ double troe_a() const { return x.troe_a; }
  __device__ __forceinline__ double troe_invT3() const { return x.troe_invT3; }
  __device__ __forceinline__ double troe_invT1() const { return x.troe_invT1; }
  __device__ __forceinline__ double troe_T2() const { return x.troe_T2; }
  __device__ __forceinline__ int has_T2() const { return x.has_T2; }
  // third-body concentration [M] = sum_k c_k + sum_e (alpha_e - 1) c_{k_e}
  template <class S, class LT>
  __device__ __forceinline__ double third_body(const MechView& m, const LT& L, double Msum) const {
    double M = Msum;
    for (int e = x.eff_begin; e < x.eff_end; ++e) M += m.eff[e].alpha_minus_1 * L[S::C + m.eff[e].k];
    return M;
  }
  // efficiency entries for the Jacobian's [M] column terms
  __device__ __forceinline__ int eff_begin() const { return x.eff_begin; }
  __device__ __forceinline__ int eff_end() const { return x.eff_end; }
  __device__ __forceinline__ int eff_k(const MechView& m, int e) const { return m.eff[e].k; }
  __device__ __forceinline__ double eff_am1(const MechView& m, int e) const { return m.eff[e].alpha_minus_1; }
};

// Troe / Lindemann blending: returns k_f and, if JAC, d ln k_f/dT (fixed [M]) and d k_f / d[M].
template <bool JAC, class XD>
__device__ __forceinline__ double falloff(const MechView& m, const XD& x, double T, double lnT, double invT,
                                          double M, double kinf, double& dlnkf, double& dkf_dM) {
  const double k0 = exp_tab(x.lnA0() + x.b0() * lnT - x.EaR0() * invT, m.exptab);
  const double Pr = k0 * M / kinf;
  double F = 1.0, D = 0.0, dlnF_T = 0.0;
  if (x.type() == RX_TROE) {
    const double e3 = exp_tab(-T * x.troe_invT3(), m.exptab), e1 = exp_tab(-T * x.troe_invT1(), m.exptab);
    double Fc = (1.0 - x.troe_a()) * e3 + x.troe_a() * e1;
    double dFc = -(1.0 - x.troe_a()) * x.troe_invT3() * e3 - x.troe_a() * x.troe_invT1() * e1;
    if (x.has_T2()) {
      const double e2 = exp_tab(-x.troe_T2() * invT, m.exptab);
      Fc += e2;
      dFc += x.troe_T2() * invT * invT * e2;
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
    const double dlnkinf = (x.b() + x.EaR() * invT) * invT;
    const double dlnk0 = (x.b0() + x.EaR0() * invT) * invT;
    const double dlnPr = dlnk0 - dlnkinf;
    dlnkf = dlnkinf + dlnF_T + D * dlnPr + dlnPr / opr;
    dkf_dM = k0 * F / opr * (D + 1.0 / opr);
  }
  return kf;
}

// Mixture quantities of one f evaluation, kept for the Jacobian assembly.
struct MixState {
  double rho, invrho, cpm, dcpm, sumYW;
  double invT, inv_cp;   // 1/T and 1/c_p (J/(kg K)) of the same evaluation
};

// Temperature-dependent quantities shared by the reaction terms of one f evaluation.
struct RhsCtx {
  double T, invT, lnT, lnPRT, Msum, RT, rho, invrho, cpm, dcpm, sumYW;
  bool poison;   // the argument makes f non-finite: f is returned as NaN
};

// Species part of f: concentrations C, G/RT, H/RT (and Cp/R), mixture properties;
// clears WDOT (and WT, D).
template <int K, bool JAC, class S, class LT>
__device__ __forceinline__ RhsCtx rhs_species(const MechView& m, const LT& L, double invp) {
  RhsCtx cx;
  // A wild stage argument (T not a positive finite number, or a mixture whose 1/rho is
  // zero, subnormal or not finite) makes f NaN.  f is then evaluated at stand-in values
  // and returned as NaN (rhs_output), so no division or logarithm takes its
  // special-value path; the attempt is rejected as non-finite either way, and every
  // other argument runs the same operations on the same values.
  const double Tin = L[S::ARG + K];
  const bool Tbad = !(Tin > 0.0) || !finite_bits(Tin);
  const double T = Tbad ? 1000.0 : Tin;
  cx.T = T;
  cx.invT = 1.0 / T;
  cx.lnT = log_tab(T, m.logtab);
  const double invT = cx.invT, lnT = cx.lnT;
  const SpecPacked* sp = m.sp;

  double sumYW = 0.0;
#pragma unroll (LT::kUnroll)
  for (int k = 0; k < K; ++k) {
    const double yw = L[S::ARG + k] * sp[k].Winv;
    L[S::C + k] = yw;
    sumYW += yw;
  }
  const double RT = kRu * T;
  const double invrho0 = RT * sumYW * invp;
  const bool rbad = !(abs_bits(invrho0) >= 0x0010000000000000ull && finite_bits(invrho0));
  const double invrho = rbad ? 1.0 : invrho0;
  cx.poison = Tbad || rbad;
  const double rho = 1.0 / invrho;
  double Msum = 0.0, cpm = 0.0, dcpm = 0.0;
#pragma unroll (LT::kUnroll)
  for (int k = 0; k < K; ++k) {
    const double yw = L[S::C + k];
    const double c = yw * rho;
    L[S::C + k] = c;
    Msum += c;
    const int r = (T >= sp[k].Tmid) ? 1 : 0;
    const double* a = sp[k].cp[r];
    const double cp = a[0] + T * (a[1] + T * (a[2] + T * (a[3] + T * a[4])));
    const double* hh = sp[k].h[r];
    const double h = hh[0] + T * (hh[1] + T * (hh[2] + T * (hh[3] + T * hh[4]))) + hh[5] * invT;
    const double* gg = sp[k].g[r];
    const double g = gg[0] + gg[1] * lnT + T * (gg[2] + T * (gg[3] + T * (gg[4] + T * gg[5]))) + gg[6] * invT;
    L[S::HRT + k] = h;
    L[S::G + k] = g;
    cpm += yw * cp;
    L[S::WDOT + k] = 0.0;
    if (JAC) {
      const double* dc = sp[k].dcp[r];
      dcpm += yw * (dc[0] + T * (dc[1] + T * (dc[2] + T * dc[3])));
      L[S::CPR + k] = cp;
      L[S::WT + k] = 0.0;
    }
  }
  if (JAC) {
#pragma unroll 1
    for (int k = 0; k < K; ++k)
#pragma unroll
      for (int j = 0; j < K; ++j) L.sm(S::MX + k * (K + 1) + j) = 0.0;
  }
  cx.lnPRT = kLnPstdOverRu - lnT;
  cx.Msum = Msum;
  cx.RT = RT;
  cx.rho = rho;
  cx.invrho = invrho;
  cx.cpm = cpm;
  cx.dcpm = dcpm;
  cx.sumYW = sumYW;
  return cx;
}

// One reaction's contribution to WDOT (and, if JAC, to WT and D).
template <int K, bool JAC, class S, class X, class LT>
__device__ __forceinline__ void reaction_term(const MechView& m, const LT& L, const RhsCtx& cx, const X& x) {
  constexpr int N = S::N;
  const double T = cx.T, invT = cx.invT, lnT = cx.lnT;
  const double lnk = x.lnA() + x.b() * lnT - x.EaR() * invT;
  double M = 1.0;
  if (x.type() != RX_ELEM) M = x.template third_body<S>(m, L, cx.Msum);
  const bool fo = (x.type() == RX_LINDEMANN || x.type() == RX_TROE);
  double kf, dlnkf = 0.0, dkf_dM = 0.0;
  if (fo) {
    kf = falloff<JAC>(m, x, T, lnT, invT, M, exp_tab(lnk, m.exptab), dlnkf, dkf_dM);
  } else {
    kf = exp_tab(lnk, m.exptab);
    if (JAC) dlnkf = (x.b() + x.EaR() * invT) * invT;
  }
  double kr = 0.0, dlnKc = 0.0;
  if (x.rev()) {
    // ln K_c = sum_reac nu' g - sum_prod nu'' g + dnu ln(P_std/(R_u T))
    double lnKc = x.dnu() * cx.lnPRT;
    double dh = 0.0;
    for (int q = 0; q < x.nf(); ++q) {
      lnKc += x.fod(q) * L[S::G + x.fi(q)];
      if (JAC) dh -= x.fod(q) * L[S::HRT + x.fi(q)];
    }
    for (int q = 0; q < x.nb(); ++q) {
      lnKc -= x.bod(q) * L[S::G + x.bi(q)];
      if (JAC) dh += x.bod(q) * L[S::HRT + x.bi(q)];
    }
    kr = fo ? kf * exp_tab(-lnKc, m.exptab) : exp_tab(lnk - lnKc, m.exptab);
    if (JAC) dlnKc = (dh - x.dnu()) * invT;
  }
  // concentration products of both sides (orders 1..3, at most three species per side)
  double cf[kMaxSide], cb[kMaxSide], pf[kMaxSide], pb[kMaxSide];
#pragma unroll
  for (int q = 0; q < kMaxSide; ++q) {
    cf[q] = (q < x.nf()) ? L[S::C + x.fi(q)] : 1.0;
    cb[q] = (q < x.nb()) ? L[S::C + x.bi(q)] : 1.0;
    pf[q] = (q < x.nf()) ? ipow(cf[q], x.fo(q)) : 1.0;
    pb[q] = (q < x.nb()) ? ipow(cb[q], x.bo(q)) : 1.0;
  }
  double Pf = pf[0], Pb = pb[0];
  if (x.nf() > 1) Pf *= pf[1];
  if (x.nf() > 2) Pf *= pf[2];
  if (x.nb() > 1) Pb *= pb[1];
  if (x.nb() > 2) Pb *= pb[2];
  const double q0 = kf * Pf - kr * Pb;
  const bool tb = (x.type() == RX_THREEBODY);
  const double q = tb ? M * q0 : q0;
  for (int pp = 0; pp < x.np(); ++pp) L[S::WDOT + x.pi(pp)] += x.pnu(pp) * q;
  if (JAC) {
    const double mf = tb ? M : 1.0;
    const double dqdT = mf * (kf * dlnkf * Pf - kr * (dlnkf - dlnKc) * Pb);
    // d q / d c for each species of each side: mf k d(prod)/dc, d(c^o)/dc = o c^(o-1)
    double gf[kMaxSide], gb[kMaxSide];
    const double mkf = mf * kf, mkr = mf * kr;
#pragma unroll
    for (int s = 0; s < kMaxSide; ++s) {
      const double df = (x.fo(s) == 1) ? 1.0 : (x.fo(s) == 2 ? 2.0 * cf[s] : 3.0 * cf[s] * cf[s]);
      const double db = (x.bo(s) == 1) ? 1.0 : (x.bo(s) == 2 ? 2.0 * cb[s] : 3.0 * cb[s] * cb[s]);
      double of = 1.0, ob = 1.0;
#pragma unroll
      for (int t = 0; t < kMaxSide; ++t) {
        if (t != s && t < x.nf()) of *= pf[t];
        if (t != s && t < x.nb()) ob *= pb[t];
      }
      gf[s] = mkf * df * of;
      gb[s] = -mkr * db * ob;
    }
    double allc = 0.0;   // d q / d [M] through the third body or falloff blending
    if (tb) allc = q0;
    else if (fo) allc = (kf != 0.0) ? dkf_dM * (q0 / kf) : 0.0;
    for (int pp = 0; pp < x.np(); ++pp) {
      const int k = x.pi(pp);
      const double nu = x.pnu(pp);
      L[S::WT + k] += nu * dqdT;
      const int row = S::MX + k * N;
      for (int s = 0; s < x.nf(); ++s) L.sm(row + x.fi(s)) += nu * gf[s];
      for (int s = 0; s < x.nb(); ++s) L.sm(row + x.bi(s)) += nu * gb[s];
      if (x.type() != RX_ELEM) {
        const double base = nu * allc;
#pragma unroll 3
        for (int j = 0; j < K; ++j) L.sm(row + j) += base;
        for (int e = x.eff_begin(); e < x.eff_end(); ++e) L.sm(row + x.eff_k(m, e)) += base * x.eff_am1(m, e);
      }
    }
  }
}

// f output (slots VEC) from WDOT.
template <int K, bool JAC, class S, class LT>
__device__ __forceinline__ MixState rhs_output(const MechView& m, const LT& L, const RhsCtx& cx) {
  const SpecPacked* sp = m.sp;
  double sum_hw = 0.0;
#pragma unroll (LT::kUnroll)
  for (int k = 0; k < K; ++k) {
    const double w = L[S::WDOT + k];
    L[S::VEC + k] = sp[k].W * w * cx.invrho;
    sum_hw += L[S::HRT + k] * w;
  }
  const double cpm_J = kRu * cx.cpm;  // J/(kg K)
  const double inv_cp = 1.0 / cpm_J;
  L[S::VEC + K] = -cx.RT * sum_hw * cx.invrho * inv_cp;
  if (cx.poison) {
    const double nan = __longlong_as_double(0x7ff8000000000000LL);
#pragma unroll
    for (int i = 0; i <= K; ++i) L[S::VEC + i] = nan;
  }
  MixState ms;
  ms.rho = cx.rho;
  ms.invrho = cx.invrho;
  ms.cpm = cpm_J;
  ms.dcpm = kRu * cx.dcpm;
  ms.sumYW = cx.sumYW;
  ms.invT = cx.invT;
  ms.inv_cp = inv_cp;
  return ms;
}

// The reactions of the mechanism image in order, each read through an RxView.
// A specialised kernel supplies its own sequence type with the same each():
// one generated descriptor per reaction, unrolled.
struct GenericReactions {
  template <class F>
  static __device__ __forceinline__ void each(const MechView& m, F&& f) {
    const int R = m.hdr->R;
#pragma unroll 1
    for (int r = 0; r < R; ++r) f(RxView{m.rx[r]}, r);
  }
};

// f over a reaction sequence RX: f at the state in slots ARG (Y_0..Y_{K-1}, T);
// result in slots VEC.  Fills C, G, HRT, WDOT and, if JAC, CPR, WT and
// D = d omega / d c (fixed T) in MX[k][j], k, j < K.
template <class RX>
struct RhsOf {
  template <int K, bool JAC, class S, class LT>
  static __device__ __forceinline__ MixState eval(const MechView& m, const LT& L, double invp) {
    const RhsCtx cx = rhs_species<K, JAC, S>(m, L, invp);
    RX::each(m, [&](const auto& x, int) { reaction_term<K, JAC, S>(m, L, cx, x); });
    return rhs_output<K, JAC, S>(m, L, cx);
  }
};

// The generic f of the thread-per-cell kernels (reactions read from the image).
using GenericRhs = RhsOf<GenericReactions>;

template <int K, bool JAC, class S = Slots<K>, class LT = Lane>
__device__ __forceinline__ MixState eval_rhs(const MechView& m, const LT& L, double invp) {
  return GenericRhs::eval<K, JAC, S>(m, L, invp);
}

// Complete the Jacobian from D (in MX) and f (in VEC), then store I/(gamma h) - J in MX.
template <int K, class S = Slots<K>, class LT = Lane>
__device__ __forceinline__ void assemble_matrix(const MechView& m, const LT& L, double T, const MixState& ms,
                                                double inv_gh, double invp) {
  constexpr int N = S::N;
  const double invT = ms.invT;
  const double RT = kRu * T;
  const double Wbar = ms.rho * RT * invp;   // p Wbar = rho R_u T: the mean molar mass without a division
  const SpecPacked* sp = m.sp;
  // D c (into G) and H^T D (into ARG)
#pragma unroll (LT::kUnrollOuter)
  for (int k = 0; k < K; ++k) {
    double acc = 0.0;
#pragma unroll
    for (int j = 0; j < K; ++j) acc += L.sm(S::MX + k * N + j) * L[S::C + j];
    L[S::G + k] = acc;
  }
#pragma unroll (LT::kUnrollOuter)
  for (int i = 0; i < K; ++i) {
    double acc = 0.0;
#pragma unroll
    for (int k = 0; k < K; ++k) acc += L[S::HRT + k] * L.sm(S::MX + k * N + i);
    L[S::ARG + i] = acc;
  }
  double HDc = 0.0, Cw = 0.0, HwT = 0.0;
#pragma unroll (LT::kUnroll)
  for (int k = 0; k < K; ++k) {
    const double Dc = L[S::G + k], h = L[S::HRT + k];
    HDc += h * Dc;
    Cw += L[S::CPR + k] * L[S::WDOT + k];
    HwT += h * (L[S::WT + k] - Dc * invT);
  }
  const double fT = L[S::VEC + K];
  // species rows: J_ki = W_k/W_i D_ki + W_k Wbar/(W_i rho) (wdot_k - Dc_k); J_kT
#pragma unroll (LT::kUnrollOuter)
  for (int k = 0; k < K; ++k) {
    const double Wk = sp[k].W;
    const double e = L[S::WDOT + k] - L[S::G + k];
    const double Bk = Wk * Wbar * e * ms.invrho;
    const int row = S::MX + k * N;
#pragma unroll
    for (int i = 0; i < K; ++i) {
      const double J = sp[i].Winv * (Wk * L.sm(row + i) + Bk);
      L.sm(row + i) = (i == k ? inv_gh : 0.0) - J;
    }
    L.sm(row + K) = -(Wk * ms.invrho * (L[S::WT + k] + e * invT));
  }
  // temperature row
  const double inv_cp = ms.inv_cp;
  const double coef = -RT * inv_cp;
  const double wHDc = Wbar * ms.invrho * HDc;
  const double fcp = fT * inv_cp;
#pragma unroll (LT::kUnroll)
  for (int i = 0; i < K; ++i) {
    const double J = sp[i].Winv * (coef * (L[S::ARG + i] - wHDc) - fcp * (kRu * L[S::CPR + i] - ms.cpm * Wbar));
    L.sm(S::MX + K * N + i) = -J;
  }
  const double JTT = -(kRu * Cw + RT * HwT) * ms.invrho * inv_cp + fT * invT - fT * ms.dcpm * inv_cp;
  L.sm(S::MX + K * N + K) = inv_gh - JTT;
}

// Compiler-only memory fence: shared-memory loads and stores are not moved across it,
// which bounds how many matrix elements the unrolled LU and solves keep in registers.
__device__ __forceinline__ void mem_fence_compiler() { asm volatile("" ::: "memory"); }

// In-place LU with partial pivoting of MX (row-major N x N, rows physically
// interchanged), fully unrolled.  On return MX holds the unit lower factor below the
// diagonal, U above it and 1/U_kk on the diagonal.  The interchanges come back as two
// words of 4-bit row indices: `swaps` (field k: the row exchanged with row k at step
// k) and `perm` (field i: the original row now at position i, so (P b)_i = b[perm_i]).
// The pivot of column k is the first row of largest |M_ik|, found by integer
// comparisons of the magnitudes' bit patterns.  The rows of a step's trailing update
// are software-pipelined: the next row's loads are issued before the current row's
// multiply-adds.  Returns false on a zero pivot.
template <int K, class LT = Lane>
__device__ __forceinline__ bool lu_factor(const LT& L, unsigned long long& swaps, unsigned long long& perm) {
  using S = Slots<K>;
  constexpr int N = S::N;
  static_assert(N <= 16, "a pivot word holds 16 rows");
  bool ok = true;
  swaps = 0ull;
  perm = 0ull;
#pragma unroll
  for (int i = 0; i < N; ++i) perm |= (unsigned long long)i << (4 * i);
#pragma unroll
  for (int k = 0; k < N; ++k) {
    int p = k;
    unsigned long long amax = abs_bits(L.sm(S::MX + k * N + k));
#pragma unroll
    for (int i = k + 1; i < N; ++i) {
      const unsigned long long v = abs_bits(L.sm(S::MX + i * N + k));
      if (v > amax) {
        amax = v;
        p = i;
      }
    }
    swaps |= (unsigned long long)p << (4 * k);
    const unsigned long long d = ((perm >> (4 * k)) ^ (perm >> (4 * p))) & 15ull;
    perm ^= (d << (4 * k)) | (d << (4 * p));
    if (amax == 0ull) ok = false;
    if (p != k) {
#pragma unroll
      for (int j = 0; j < N; ++j) {
        const double t = L.sm(S::MX + k * N + j);
        L.sm(S::MX + k * N + j) = L.sm(S::MX + p * N + j);
        L.sm(S::MX + p * N + j) = t;
      }
    }
    mem_fence_compiler();
    const double inv = 1.0 / L.sm(S::MX + k * N + k);
    L.sm(S::MX + k * N + k) = inv;
    if (k + 1 < N) {
      double u[N], r[N];
#pragma unroll
      for (int j = k + 1; j < N; ++j) u[j] = L.sm(S::MX + k * N + j);
#pragma unroll
      for (int j = k; j < N; ++j) r[j] = L.sm(S::MX + (k + 1) * N + j);
#pragma unroll
      for (int i = k + 1; i < N; ++i) {
        double rn[N];
        if (i + 1 < N) {
#pragma unroll
          for (int j = k; j < N; ++j) rn[j] = L.sm(S::MX + (i + 1) * N + j);
        }
        mem_fence_compiler();
        const double l = r[k] * inv;
        L.sm(S::MX + i * N + k) = l;
#pragma unroll
        for (int j = k + 1; j < N; ++j) L.sm(S::MX + i * N + j) = r[j] - l * u[j];
        if (i + 1 < N) {
#pragma unroll
          for (int j = k; j < N; ++j) r[j] = rn[j];
        }
      }
    }
    mem_fence_compiler();
  }
  return ok;
}

// Solve M x = b with the factors of lu_factor: b is read from slots VEC (original row
// order, gathered through `perm`) and x is returned in registers.  Both substitutions
// are column oriented: once a component is final it updates every later one, so the
// multiply-adds of a column are independent of one another; the next column's factor
// entries are loaded while the current column is applied.
template <int K, class LT = Lane>
__device__ __forceinline__ void lu_solve(const LT& L, unsigned long long perm, double (&x)[K + 1]) {
  using S = Slots<K>;
  constexpr int N = S::N;
  if constexpr (LT::kRegs) {
    // register-resident right-hand side: gather (P b)_i through a small per-thread
    // array (local memory, L1), which keeps the code short
    double b[N];
#pragma unroll
    for (int j = 0; j < N; ++j) b[j] = L[S::VEC + j];
#pragma unroll
    for (int i = 0; i < N; ++i) x[i] = b[(int)((perm >> (4 * i)) & 15ull)];
  } else {
#pragma unroll
    for (int i = 0; i < N; ++i) x[i] = L[S::VEC + (int)((perm >> (4 * i)) & 15ull)];
  }
  double c[N], cn[N];
  // forward substitution with the unit lower factor, column j = 0 .. N-2
#pragma unroll
  for (int i = 1; i < N; ++i) c[i] = L.sm(S::MX + i * N + 0);
#pragma unroll
  for (int j = 0; j < N - 1; ++j) {
    if (j + 1 < N - 1) {
#pragma unroll
      for (int i = j + 2; i < N; ++i) cn[i] = L.sm(S::MX + i * N + (j + 1));
    }
    mem_fence_compiler();
#pragma unroll
    for (int i = j + 1; i < N; ++i) x[i] -= c[i] * x[j];
#pragma unroll
    for (int i = j + 2; i < N; ++i) c[i] = cn[i];
  }
  // back substitution with U (1/U_kk on the diagonal), column j = N-1 .. 0
#pragma unroll
  for (int i = 0; i < N; ++i) c[i] = L.sm(S::MX + i * N + (N - 1));
#pragma unroll
  for (int j = N - 1; j >= 0; --j) {
    if (j > 0) {
#pragma unroll
      for (int i = 0; i < j; ++i) cn[i] = L.sm(S::MX + i * N + (j - 1));
    }
    mem_fence_compiler();
    x[j] *= c[j];
#pragma unroll
    for (int i = 0; i < j; ++i) x[i] -= c[i] * x[j];
#pragma unroll
    for (int i = 0; i < j; ++i) c[i] = cn[i];
  }
}

// RMS error norm of reading (g): sqrt(mean_i (e_i / (atol + rtol max(|y_i|, |yn_i|)))^2);
// `finite` reports whether every yn_i is finite (if not, the norm is not computed and 0
// is returned: the controller rejects such a candidate with facmin whatever the norm).
// The maxima and finiteness tests run on
// the integer pipe; the quotients of two components share one division, 1/(sc_a sc_b),
// unless that product leaves the normal range (then each is divided on its own).
template <int N>
__device__ __forceinline__ double error_norm(const double (&y)[N], const double (&yn)[N], const double (&e)[N],
                                             double rtol, double atol, bool& finite) {
  double sc[N];
  finite = true;
#pragma unroll
  for (int i = 0; i < N; ++i) {
    const unsigned long long a = abs_bits(y[i]), b = abs_bits(yn[i]);
    sc[i] = atol + rtol * __longlong_as_double((long long)(a > b ? a : b));
    finite = finite && finite_bits(yn[i]);
  }
  if (!finite) return 0.0;   // a non-finite candidate is rejected whatever the norm
  double sum = 0.0;
#pragma unroll
  for (int i = 0; i + 1 < N; i += 2) {
    const double pr = sc[i] * sc[i + 1];
    double q0, q1;
    if (abs_bits(pr) >= 0x0010000000000000ull && finite_bits(pr)) {
      const double inv = 1.0 / pr;
      q0 = e[i] * (sc[i + 1] * inv);
      q1 = e[i + 1] * (sc[i] * inv);
    } else {
      q0 = e[i] / sc[i];
      q1 = e[i + 1] / sc[i + 1];
    }
    sum += q0 * q0;
    sum += q1 * q1;
  }
  if (N & 1) {
    const double q = e[N - 1] / sc[N - 1];
    sum += q * q;
  }
  return sqrt(sum / N);
}

// One Rosenbrock attempt (RODAS3, or ROS2 with METHOD = kMethodRos2) of size h from y,
// the arithmetic every thread-per-cell kernel that integrates shares (the forward
// step, and the adjoint's re-integration, which must retrace the forward's steps
// bit for bit):
//   f(y) and J(y); M = I/(gamma h) - J factorised in place; the stages
//   M u_i = f(y + sum_j a_ij u_j) + sum_j (c_ij/h) u_j; yn = y + sum_i m_i u_i;
//   err = RMS norm of the embedded estimate (error_norm).
// Returns false on a zero pivot (the cell fails with RDE_CELL_LU_SINGULAR), else true.  On return the lane slots
// hold the factors of M (lu_factor's layout) and `swaps` their interchanges; with
// STAGES the stage vectors u_1..u_4 are copied to U (RODAS3).
template <int K, class RHS, int METHOD, bool STAGES = false, class LT = Lane>
__device__ __forceinline__ bool rosenbrock_attempt(const MechView& m, const LT& L, double invp, const double (&y)[K + 1],
                                                  double h, const Opts& o, double (&yn)[K + 1], double& err,
                                                  bool& finite, unsigned long long& swaps, double (&U)[4][K + 1]) {
  using S = Slots<K>;
  constexpr int N = K + 1;
  constexpr double gamma = METHOD == kMethodRos2 ? kR2Gamma : kGamma;
#pragma unroll
  for (int i = 0; i < N; ++i) L[S::ARG + i] = y[i];
  const MixState ms = RHS::template eval<K, true, S>(m, L, invp);
  double f0[N];
#pragma unroll
  for (int i = 0; i < N; ++i) f0[i] = L[S::VEC + i];
  const double invh = 1.0 / h;
  assemble_matrix<K>(m, L, y[K], ms, (1.0 / gamma) * invh, invp);
  unsigned long long perm;
  if (!lu_factor<K>(L, swaps, perm)) return false;
  double ev[N];   // the embedded error estimate
  if constexpr (METHOD == kMethodRos2) {
    double u1[N], u2[N];
    // stage 1: M u1 = f(y)   (the slots VEC still hold f(y))
    lu_solve<K>(L, perm, u1);
#pragma unroll
    for (int i = 0; i < N; ++i) L[S::ARG + i] = y[i] + kR2A21 * u1[i];
    // stage 2: M u2 = f(y + a21 u1) + (c21/h) u1
    RHS::template eval<K, false, S>(m, L, invp);
    const double c21h = kR2C21 * invh;
#pragma unroll
    for (int i = 0; i < N; ++i) L[S::VEC + i] += c21h * u1[i];
    lu_solve<K>(L, perm, u2);
#pragma unroll
    for (int i = 0; i < N; ++i) {
      yn[i] = y[i] + kR2M1 * u1[i] + kR2M2 * u2[i];
      ev[i] = kR2E * (u1[i] + u2[i]);
    }
  } else {
    double u1[N], u2[N], u3[N], u4[N];
    // stage 1: M u1 = f(y)   (the slots VEC still hold f(y))
    lu_solve<K>(L, perm, u1);
    // stage 2: M u2 = f(y) + (c21/h) u1
    const double c21h = kC21 * invh;
#pragma unroll
    for (int i = 0; i < N; ++i) L[S::VEC + i] = f0[i] + c21h * u1[i];
    lu_solve<K>(L, perm, u2);
#pragma unroll
    for (int i = 0; i < N; ++i) {
      u3[i] = 0.0;
      u4[i] = 0.0;
    }
    // stages 3 and 4 share one body: M u = f(y + 2 u1 + a43 u3) + (u1 - u2 + c43 u3)/h
#pragma unroll 1
    for (int st = 0; st < 2; ++st) {
#pragma unroll
      for (int i = 0; i < N; ++i) L[S::ARG + i] = y[i] + 2.0 * u1[i] + u3[i];
      RHS::template eval<K, false, S>(m, L, invp);
      const double c3 = st ? kC43 : 0.0;
#pragma unroll
      for (int i = 0; i < N; ++i) L[S::VEC + i] += invh * (u1[i] - u2[i] + c3 * u3[i]);
      double w[N];
      lu_solve<K>(L, perm, w);
#pragma unroll
      for (int i = 0; i < N; ++i) {
        u3[i] = st ? u3[i] : w[i];
        u4[i] = st ? w[i] : u4[i];
      }
    }
    // y_new = (y + 2 u1 + u3) + u4 (the stage-4 argument is still in ARG); error = u4
#pragma unroll
    for (int i = 0; i < N; ++i) {
      yn[i] = L[S::ARG + i] + u4[i];
      ev[i] = u4[i];
    }
    if constexpr (STAGES) {
#pragma unroll
      for (int i = 0; i < N; ++i) {
        U[0][i] = u1[i];
        U[1][i] = u2[i];
        U[2][i] = u3[i];
        U[3][i] = u4[i];
      }
    }
  }
  err = error_norm<N>(y, yn, ev, o.rtol, o.atol, finite);
  return true;
}

// One step of the extrapolation method (kMethodExtrap) of size h from y.  The three
// matrices I/h_j - J share J: the Jacobian is assembled once as -J (1/(gamma h) = 0),
// parked in the lane's slice of a global scratch (Jg[e * nl], N^2 doubles, coalesced
// across lanes), and each I/h_j - J is rebuilt from it (a diagonal update) before its
// factorisation.  Per step: one f + Jacobian, three more f, three LU, six solves.
// Returns false on a zero pivot; err and finite as rosenbrock_attempt.
template <int K, class RHS, class LT = Lane>
__device__ __forceinline__ bool extrapolation_attempt(const MechView& m, const LT& L, double invp,
                                                      const double (&y)[K + 1], double h, const Opts& o,
                                                      double (&yn)[K + 1], double& err, bool& finite,
                                                      double* Jg, long long nl) {
  using S = Slots<K>;
  constexpr int N = K + 1;
#pragma unroll
  for (int i = 0; i < N; ++i) L[S::ARG + i] = y[i];
  const MixState ms = RHS::template eval<K, true, S>(m, L, invp);
  double f0[N];
#pragma unroll
  for (int i = 0; i < N; ++i) f0[i] = L[S::VEC + i];
  assemble_matrix<K>(m, L, y[K], ms, 0.0, invp);          // MX = -J
#pragma unroll 4
  for (int e = 0; e < N * N; ++e) Jg[e * nl] = L.sm(S::MX + e);
  const double invh = 1.0 / h;
  double T1[N], T2[N], T3[N];
#pragma unroll 1
  for (int j = 0; j < 3; ++j) {
    const double invhj = (double)(j + 1) * invh;          // 1 / (h / n_j)
    if (j > 0) {
#pragma unroll 4
      for (int e = 0; e < N * N; ++e) L.sm(S::MX + e) = Jg[e * nl];
    }
#pragma unroll
    for (int i = 0; i < N; ++i) L.sm(S::MX + i * N + i) += invhj;
    unsigned long long swaps, perm;
    if (!lu_factor<K>(L, swaps, perm)) return false;
    double yi[N];
#pragma unroll
    for (int i = 0; i < N; ++i) {
      yi[i] = y[i];
      L[S::VEC + i] = f0[i];
    }
#pragma unroll 1
    for (int sub = 0; sub <= j; ++sub) {
      if (sub > 0) {
#pragma unroll
        for (int i = 0; i < N; ++i) L[S::ARG + i] = yi[i];
        RHS::template eval<K, false, S>(m, L, invp);    // f(y_sub) into VEC
      }
      double d[N];
      lu_solve<K>(L, perm, d);
#pragma unroll
      for (int i = 0; i < N; ++i) yi[i] += d[i];
    }
#pragma unroll
    for (int i = 0; i < N; ++i) {
      T1[i] = (j == 0) ? yi[i] : T1[i];
      T2[i] = (j == 1) ? yi[i] : T2[i];
      T3[i] = (j == 2) ? yi[i] : T3[i];
    }
  }
  double ev[N];
#pragma unroll
  for (int i = 0; i < N; ++i) {
    const double t21 = T2[i] + (T2[i] - T1[i]);
    const double t31 = T3[i] + 2.0 * (T3[i] - T2[i]);
    const double t32 = t31 + (t31 - t21) * 0.5;
    yn[i] = t32;
    ev[i] = t32 - t31;
  }
  err = error_norm<N>(y, yn, ev, o.rtol, o.atol, finite);
  return true;
}

// A lane's park area in global memory (L2): element e at p[e * stride], four vectors
// of N: the cell state y, then u_1, u_2, u_3 of the current attempt.  The accesses are
// opaque to the compiler, so values parked across an f evaluation do not occupy
// registers there.
struct Park {
  double* p;
  long long stride;
  __device__ __forceinline__ void st(int e, double v) const {
    asm volatile("st.global.cg.f64 [%0], %1;" ::"l"(p + e * stride), "d"(v) : "memory");
  }
  __device__ __forceinline__ double ld(int e) const {
    double v;
    asm volatile("ld.global.cg.f64 %0, [%1];" : "=d"(v) : "l"(p + e * stride) : "memory");
    return v;
  }
};

// RODAS3 attempt of the wide kernels: the operations of rosenbrock_attempt (METHOD =
// kMethodRodas3) in the same order, with the cell state read from the park area and
// u_1..u_3 parked there across the f evaluations of stages 3 and 4 (their arguments and
// right-hand sides are rebuilt from the parked values by the same expressions).  The
// results agree with rosenbrock_attempt's to rounding: with the slots in registers the
// compiler contracts multiply-adds differently.
template <int K, class RHS, class LT>
__device__ __forceinline__ bool rodas3_attempt_parked(const MechView& m, const LT& L, double invp, const Park& P,
                                                     double h, const Opts& o, double (&yn)[K + 1], double& err,
                                                     bool& finite) {
  using S = Slots<K>;
  constexpr int N = K + 1;
  double T0;
  {
#pragma unroll
    for (int i = 0; i < N; ++i) L[S::ARG + i] = P.ld(i);
    T0 = L[S::ARG + K];
  }
  const MixState ms = RHS::template eval<K, true, S>(m, L, invp);
  double f0[N];
#pragma unroll
  for (int i = 0; i < N; ++i) f0[i] = L[S::VEC + i];
  const double invh = 1.0 / h;
  assemble_matrix<K>(m, L, T0, ms, (1.0 / kGamma) * invh, invp);
  unsigned long long swaps, perm;
  if (!lu_factor<K>(L, swaps, perm)) return false;
  {
    double u1[N], u2[N];
    // stage 1: M u1 = f(y)   (the slots VEC still hold f(y))
    lu_solve<K>(L, perm, u1);
    // stage 2: M u2 = f(y) + (c21/h) u1
    const double c21h = kC21 * invh;
#pragma unroll
    for (int i = 0; i < N; ++i) L[S::VEC + i] = f0[i] + c21h * u1[i];
    lu_solve<K>(L, perm, u2);
#pragma unroll
    for (int i = 0; i < N; ++i) {
      P.st(N + i, u1[i]);
      P.st(2 * N + i, u2[i]);
      P.st(3 * N + i, 0.0);
    }
  }
  double u4[N];
  // stages 3 and 4: M u = f(y + 2 u1 + a43 u3) + (u1 - u2 + c43 u3)/h
#pragma unroll 1
  for (int st = 0; st < 2; ++st) {
#pragma unroll
    for (int i = 0; i < N; ++i) L[S::ARG + i] = P.ld(i) + 2.0 * P.ld(N + i) + P.ld(3 * N + i);
    RHS::template eval<K, false, S>(m, L, invp);
    const double c3 = st ? kC43 : 0.0;
#pragma unroll
    for (int i = 0; i < N; ++i) L[S::VEC + i] += invh * (P.ld(N + i) - P.ld(2 * N + i) + c3 * P.ld(3 * N + i));
    double w[N];
    lu_solve<K>(L, perm, w);
    if (st == 0) {
#pragma unroll
      for (int i = 0; i < N; ++i) P.st(3 * N + i, w[i]);
    } else {
#pragma unroll
      for (int i = 0; i < N; ++i) u4[i] = w[i];
    }
  }
  // y_new = (y + 2 u1 + u3) + u4; error = u4
  double y[N];
#pragma unroll
  for (int i = 0; i < N; ++i) {
    y[i] = P.ld(i);
    yn[i] = (y[i] + 2.0 * P.ld(N + i) + P.ld(3 * N + i)) + u4[i];
  }
  err = error_norm<N>(y, yn, u4, o.rtol, o.atol, finite);
  return true;
}

// Step-size factor of the controller (reading (h)): after an accepted attempt
// min(facmax', max(facmin, safety err^(-1/(q+1)))) with facmax' = 1 right after a
// rejection; after a rejected one max(facmin, safety err^(-1/(q+1))), or facmin for a
// non-finite attempt.  q = 2 (RODAS3) or 1 (ROS2).
template <int METHOD>
__device__ __forceinline__ double step_factor(double err, bool finite, bool accepted, bool reject_prev,
                                              const Opts& o) {
  const double rroot = !finite ? 1.0 : (METHOD == kMethodRos2 ? rsqrt(err) : rcbrt(err));   // unused if !finite
  if (accepted) return fmin(reject_prev ? 1.0 : o.facmax, fmax(o.facmin, o.safety * rroot));
  return (finite && isfinite(err)) ? fmax(o.facmin, o.safety * rroot) : o.facmin;
}

}  // namespace rde
