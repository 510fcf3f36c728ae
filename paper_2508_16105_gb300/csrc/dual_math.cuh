// Dual numbers (a value and its derivative along one direction) and the scalar
// helpers of the chemistry terms written once for double and Dual: the table-
// driven exp / log, integer powers and the falloff blend with its derivatives.
// Shared by the discrete adjoint's thread-per-cell and CTA-per-cell kernels.
#pragma once
#include "chem_device.cuh"

namespace rde {

// ---------------------------------------------------------------------------
// dual numbers: value and derivative along one direction
// ---------------------------------------------------------------------------
struct Dual {
  double v, d;
};
__device__ __forceinline__ Dual mk(double v, double d) { return Dual{v, d}; }
__device__ __forceinline__ Dual operator+(Dual a, Dual b) { return mk(a.v + b.v, a.d + b.d); }
__device__ __forceinline__ Dual operator-(Dual a, Dual b) { return mk(a.v - b.v, a.d - b.d); }
__device__ __forceinline__ Dual operator-(Dual a) { return mk(-a.v, -a.d); }
__device__ __forceinline__ Dual operator+(Dual a, double b) { return mk(a.v + b, a.d); }
__device__ __forceinline__ Dual operator+(double a, Dual b) { return mk(a + b.v, b.d); }
__device__ __forceinline__ Dual operator-(Dual a, double b) { return mk(a.v - b, a.d); }
__device__ __forceinline__ Dual operator-(double a, Dual b) { return mk(a - b.v, -b.d); }
__device__ __forceinline__ Dual operator*(Dual a, Dual b) { return mk(a.v * b.v, fma(a.v, b.d, a.d * b.v)); }
__device__ __forceinline__ Dual operator*(double a, Dual b) { return mk(a * b.v, a * b.d); }
__device__ __forceinline__ Dual operator*(Dual a, double b) { return mk(a.v * b, a.d * b); }
__device__ __forceinline__ Dual operator/(Dual a, Dual b) {
  const double inv = 1.0 / b.v, q = a.v * inv;
  return mk(q, (a.d - q * b.d) * inv);
}
__device__ __forceinline__ Dual operator/(double a, Dual b) {
  const double inv = 1.0 / b.v, q = a * inv;
  return mk(q, -q * b.d * inv);
}
__device__ __forceinline__ Dual operator/(Dual a, double b) { return mk(a.v / b, a.d / b); }
__device__ __forceinline__ Dual& operator+=(Dual& a, Dual b) { a = a + b; return a; }
__device__ __forceinline__ Dual& operator-=(Dual& a, Dual b) { a = a - b; return a; }
__device__ __forceinline__ Dual& operator*=(Dual& a, Dual b) { a = a * b; return a; }

__device__ __forceinline__ double val(double x) { return x; }
__device__ __forceinline__ double val(Dual x) { return x.v; }
__device__ __forceinline__ double der(double) { return 0.0; }
__device__ __forceinline__ double der(Dual x) { return x.d; }
template <class S> __device__ __forceinline__ S cst(double v);
template <> __device__ __forceinline__ double cst<double>(double v) { return v; }
template <> __device__ __forceinline__ Dual cst<Dual>(double v) { return mk(v, 0.0); }

__device__ __forceinline__ double sexp(const MechView& m, double x) { return exp_tab(x, m.exptab); }
__device__ __forceinline__ Dual sexp(const MechView& m, Dual x) {
  const double e = exp_tab(x.v, m.exptab);
  return mk(e, e * x.d);
}
__device__ __forceinline__ double slog(const MechView& m, double x) { return log_tab(x, m.logtab); }
__device__ __forceinline__ Dual slog(const MechView& m, Dual x) { return mk(log_tab(x.v, m.logtab), x.d / x.v); }
__device__ __forceinline__ double smax300(double x) { return fmax(x, 1e-300); }
__device__ __forceinline__ Dual smax300(Dual x) { return x.v > 1e-300 ? x : mk(1e-300, 0.0); }

template <class S>
__device__ __forceinline__ S ipow_s(S c, int e) {
  S r = c;
  if (e >= 2) r = r * c;
  if (e >= 3) r = r * c;
  return r;
}

// Falloff blend with d ln k_f / dT (fixed [M]), d k_f / d[M] and phi = d ln k_f / d ln k_inf.
template <class S, class XD>
__device__ __forceinline__ S falloff_s(const MechView& m, const XD& x, S T, S lnT, S invT, S M, S kinf,
                                       S& dlnkf, S& dkf_dM, S& phi) {
  const S k0 = sexp(m, x.lnA0() + x.b0() * lnT - x.EaR0() * invT);
  const S Pr = k0 * M / kinf;
  S F = cst<S>(1.0), D = cst<S>(0.0), dlnF_T = cst<S>(0.0);
  if (x.type() == RX_TROE) {
    const S e3 = sexp(m, -(T * x.troe_invT3())), e1 = sexp(m, -(T * x.troe_invT1()));
    S Fc = (1.0 - x.troe_a()) * e3 + x.troe_a() * e1;
    S dFc = (-(1.0 - x.troe_a()) * x.troe_invT3()) * e3 - (x.troe_a() * x.troe_invT1()) * e1;
    if (x.has_T2()) {
      const S e2 = sexp(m, -(x.troe_T2() * invT));
      Fc += e2;
      dFc += x.troe_T2() * (invT * invT) * e2;
    }
    const S Lc = slog(m, Fc) * kInvLn10;
    const S cc = -0.4 - 0.67 * Lc, nn = 0.75 - 1.27 * Lc;
    const double dd = 0.14;
    const S Lp = slog(m, smax300(Pr)) * kInvLn10;
    const S u = Lp + cc, den = nn - dd * u, X = u / den;
    const S opx = 1.0 + X * X;
    F = sexp(m, kLn10 * (Lc / opx));
    const S dLc = dFc / (Fc * kLn10);
    const S dX_du = nn / (den * den);
    const S common = -(Lc * 2.0 * X) / (opx * opx);
    D = common * dX_du;
    const S du_dT = -0.67 * dLc, dn_dT = -1.27 * dLc;
    const S dX_dT = (du_dT * den - u * (dn_dT - dd * du_dT)) / (den * den);
    dlnF_T = kLn10 * (dLc / opx + common * dX_dT);
  }
  const S opr = 1.0 + Pr;
  const S kf = kinf * Pr / opr * F;
  const S dlnkinf = (x.b() + x.EaR() * invT) * invT;
  const S dlnk0 = (x.b0() + x.EaR0() * invT) * invT;
  const S dlnPr = dlnk0 - dlnkinf;
  dlnkf = dlnkinf + dlnF_T + D * dlnPr + dlnPr / opr;
  dkf_dM = k0 * F / opr * (D + 1.0 / opr);
  phi = Pr / opr - D;
  return kf;
}

}  // namespace rde
