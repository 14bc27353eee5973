// FP64 elementary functions tuned for B300's narrow FP64 pipe.
//
// On this part an FP64 FMA issues at 1/73 of the FP32 rate and CUDA's FP64
// exp / sqrt / reciprocal occupy the FP64 pipe for about 20 / 12 / 7 FMA slots.
// The functions below reach full double accuracy (a few ulp) with fewer slots:
//
//  exp_tab   table-driven exponential after P. T. P. Tang, "Table-driven
//            implementation of the exponential function in IEEE floating-point
//            arithmetic", ACM TOMS 15 (1989): x = (64 m + j) ln2/64 + r with
//            |r| <= ln2/128, exp(x) = 2^m 2^(j/64) exp(r), exp(r) by its Taylor
//            polynomial of degree 5 (truncation < 4e-17), the reduction by FMA
//            against a two-part ln2/64 (Cody-Waite), 2^m applied to the exponent
//            field.  About 10 FP64 slots.
//  rcp_nr    hardware reciprocal approximation (rcp.approx.ftz.f64, ~2^-20)
//            refined by two Newton-Raphson steps t <- t + t (1 - y t).
//  rsqrt_nr  hardware rsqrt approximation refined by two Newton-Raphson steps
//            y <- y + y (1 - s y^2) / 2.
// The reduction constants are ln2/64 split into double hi/lo parts and 64/ln2,
// evaluated to 200 bits; the table holds 2^(j/64) rounded to double.
#pragma once

#include <cstdint>

namespace lrdmc {

constexpr int EXP_TAB = 64;
constexpr double EXP_INV_L = 0x1.71547652b82fep+6;    // 64 / ln 2
constexpr double EXP_L_HI = 0x1.62e42fefa39efp-7;     // ln 2 / 64, leading double
constexpr double EXP_L_LO = 0x1.abc9e3b39803fp-62;    // ln 2 / 64 - EXP_L_HI
constexpr double EXP_SHIFTER = 0x1.8p52;              // 1.5 * 2^52: rounds to an integer

// exp(x) for x in [-700, 700]; 0 below -700 (true value < 1e-304), +inf above.
__device__ __forceinline__ double exp_tab(double x, const double* __restrict__ T) {
  const double t = fma(x, EXP_INV_L, EXP_SHIFTER);
  const int k = (int)__double2loint(t);                 // round(x * 64/ln2), two's complement
  const double kd = t - EXP_SHIFTER;
  double r = fma(kd, -EXP_L_HI, x);
  r = fma(kd, -EXP_L_LO, r);
  double q = fma(r, 1.0 / 120.0, 1.0 / 24.0);
  q = fma(r, q, 1.0 / 6.0);
  q = fma(r, q, 0.5);
  q = fma(r, q, 1.0);
  const double p = r * q;                               // exp(r) - 1
  const double tj = T[k & (EXP_TAB - 1)];
  double y = fma(tj, p, tj);
  y = __longlong_as_double(__double_as_longlong(y) + ((long long)(k >> 6) << 52));
  y = x < -700.0 ? 0.0 : y;
  return x > 700.0 ? __longlong_as_double(0x7ff0000000000000ll) : y;
}

__device__ __forceinline__ double rcp_approx(double x) {
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
  return r;
}

__device__ __forceinline__ double rsqrt_approx(double x) {
  double r;
  asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
  return r;
}

// 1/y for finite y != 0 (normal range).
__device__ __forceinline__ double rcp_nr(double y) {
  double t = rcp_approx(y);
  double e = fma(-y, t, 1.0);
  t = fma(t, e, t);
  e = fma(-y, t, 1.0);
  return fma(t, e, t);
}

// 1/sqrt(s) for s > 0 (normal range).
__device__ __forceinline__ double rsqrt_nr(double s) {
  double y = rsqrt_approx(s);
  double e = fma(-s, y * y, 1.0);
  y = fma(y * e, 0.5, y);
  e = fma(-s, y * y, 1.0);
  return fma(y * e, 0.5, y);
}

}  // namespace lrdmc
