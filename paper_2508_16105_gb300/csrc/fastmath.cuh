// Table-driven FP64 exp and log (after P. T. P. Tang, ACM TOMS 15(2), 1989 for
// exp and 16(4), 1990 for log), written for GB300, where an FP64 fused
// multiply-add is the scarce operation (two per SM per clock) and integer,
// select and shared-memory work is nearly free.
//
//   exp: x = k ln2/1024 + r, |r| <= ln2/2048;  e^x = 2^(k>>10) * T[k & 1023] * e^r,
//        T[j] = 2^(j/1024), e^r - 1 by its degree-4 Taylor polynomial
//        (truncation below 4e-20).  9 FP64 operations; error about 1 ulp.
//   log: x = 2^e m, m in [1,2);  ln x = e ln2 + logc_j + ln(m invc_j), with
//        invc_j ~ 1/c_j for the centre c_j of m's 1/128 interval and
//        ln(1+r) by its degree-7 Taylor polynomial (|r| < 2^-8.9, truncation
//        below 3e-20).  11 FP64 operations; error about 1 ulp of ln x away from
//        x = 1 (absolute error below 5e-17 within 1 % of 1).
//
// Arguments outside the fast ranges take short inline paths through the same cores
// (no library call, so a lane in a wild Rosenbrock stage costs its warp a few
// instructions, not a call that saves the register file): exp for |x| > 707 runs the
// same reduction and applies its power of two in two parts (overflow to inf, gradual
// underflow to 0; the argument is clamped to [-1060, 800] first, NaN returns NaN); log of a
// subnormal x is ln(x 2^54) - 54 ln 2, log(0) = -inf, log(inf) = inf, log of a
// negative number or NaN is NaN.  The range tests compare bit patterns (integer
// operations).  The code uses only explicit fma and exact bit operations, so host and
// device give identical bits.
#pragma once
#if !defined(__CUDACC_RTC__)  /* run-time compilation: math built in */
#include <math.h>
#include <stdint.h>
#include <string.h>
#endif

#include "fastmath_tables.h"

namespace rde {

#if defined(__CUDACC__)
#define RDE_FM __host__ __device__ __forceinline__
#else
#define RDE_FM inline
#endif

RDE_FM int64_t dbl_bits(double x) {
#if defined(__CUDA_ARCH__)
  return __double_as_longlong(x);
#else
  int64_t b;
  memcpy(&b, &x, 8);
  return b;
#endif
}

RDE_FM double bits_dbl(int64_t b) {
#if defined(__CUDA_ARCH__)
  return __longlong_as_double(b);
#else
  double x;
  memcpy(&x, &b, 8);
  return x;
#endif
}

// Fast-range tests on the bit patterns (integer operations only):
//   exp: |x| <= 707 (false for NaN);  log: x a positive normal finite number.
constexpr int64_t kBits707 = 0x4086180000000000LL;   // the bits of 707.0
RDE_FM bool exp_in_range(double x) {
  return (uint64_t)(dbl_bits(x) & 0x7fffffffffffffffLL) <= (uint64_t)kBits707;
}
RDE_FM bool log_in_range(double x) {
  return (uint64_t)(dbl_bits(x) - 0x0010000000000000LL) <= (uint64_t)(0x7fefffffffffffffLL - 0x0010000000000000LL);
}

// The table-driven evaluation with its power of two lowered by 2^bias (the reduction
// is exact for |x| <= 800; bias 0 is the fast path of exp_tab, no test, no branch).
RDE_FM double exp_tab_core_b(double x, const double* tab, int bias) {
  const double shifter = 0x1.8p52;
  const double t = fma(x, kExpLog2e1024, shifter);   // low word of t = k = nearest(x 1024/ln2)
  const double kd = t - shifter;
  double r = fma(kd, -kExpLn2Hi, x);
  r = fma(kd, -kExpLn2Lo, r);
  const int32_t k = (int32_t)(uint32_t)(uint64_t)dbl_bits(t);
  const double T = tab[k & 1023];
  double a = fma(r, 1.0 / 24.0, 1.0 / 6.0);
  a = fma(a, r, 0.5);
  const double em1 = fma(a, r * r, r);               // e^r - 1
  const double res = fma(T, em1, T);                 // in [0.9996, 2.0004): a normal number
  return bits_dbl(dbl_bits(res) + ((int64_t)((k >> 10) - bias) << 52));
}

RDE_FM double exp_tab_core(double x, const double* tab) { return exp_tab_core_b(x, tab, 0); }

// e^x outside |x| <= 707 (x clamped to [-1060, 800]): the core with its power of two
// lowered by 2^(+-512), then one multiplication by 2^(+-512), which rounds once into
// the subnormal range or overflows to inf
RDE_FM double exp_tab_wide(double x, const double* tab) {
  if (x != x) return x;
  const bool up = x > 0.0;
  const double xc = up ? fmin(x, 800.0) : fmax(x, -1060.0);
  return exp_tab_core_b(xc, tab, up ? 512 : -512) * (up ? 0x1p512 : 0x1p-512);
}

// e^x; tab = the 1024 values 2^(j/1024)
RDE_FM double exp_tab(double x, const double* tab) {
  if (!exp_in_range(x)) return exp_tab_wide(x, tab);
  return exp_tab_core(x, tab);
}

// Fast path of log_tab for a positive normal finite argument (no test, no branch).
RDE_FM double log_tab_core(double x, const double* tab) {
  const int64_t b = dbl_bits(x);
  const int e = (int)(b >> 52) - 1023;
  const int j = (int)((b >> 45) & 127);
  const double m = bits_dbl((b & 0x000fffffffffffffLL) | 0x3ff0000000000000LL);
  const double r = fma(m, tab[2 * j], -1.0);
  double p = fma(r, 1.0 / 7.0, -1.0 / 6.0);
  p = fma(p, r, 0.2);
  p = fma(p, r, -0.25);
  p = fma(p, r, 1.0 / 3.0);
  p = fma(p, r, -0.5);
  const double l1p = fma(p, r * r, r);               // ln(1 + r)
  const double ed = (double)e;
  const double hi = fma(ed, kLogLn2Hi, tab[2 * j + 1]);
  return hi + fma(ed, kLogLn2Lo, l1p);
}

// ln x outside the positive normal finite numbers
RDE_FM double log_tab_wide(double x, const double* tab) {
  if (x > 0.0 && x < 0x1p-1022) return log_tab_core(x * 0x1p54, tab) - kLog54Ln2;   // subnormal
  if (x == 0.0) return bits_dbl((int64_t)0xfff0000000000000ULL);                   // -inf
  if (x > 0.0) return x;                                                              // +inf
  return bits_dbl(0x7ff8000000000000LL);                                              // negative, NaN
}

// ln x; tab = 128 pairs (invc_j, logc_j = -ln invc_j)
RDE_FM double log_tab(double x, const double* tab) {
  if (!log_in_range(x)) return log_tab_wide(x, tab);
  return log_tab_core(x, tab);
}

}  // namespace rde
