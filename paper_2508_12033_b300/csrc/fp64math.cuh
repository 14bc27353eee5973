// FP64 elementary functions tuned for B300's narrow FP64 pipe.
//
// On this part an FP64 FMA issues at 1/73 of the FP32 rate and CUDA's FP64
// exp / sqrt / reciprocal occupy the FP64 pipe for about 20 / 12 / 7 FMA slots.
// The functions below reach full double accuracy (a few ulp) with fewer slots:
//
//  exp_tab   table-driven exponential after P. T. P. Tang, "Table-driven
//            implementation of the exponential function in IEEE floating-point
//            arithmetic", ACM TOMS 15 (1989), with a 256-entry table:
//            x = (256 m + j) ln2/256 + r with |r| <= ln2/512, exp(x) =
//            2^m 2^(j/256) exp(r), exp(r) - 1 by its Taylor polynomial of degree 4
//            (truncation |r|^5/120 < 4e-17), the reduction by FMA against a
//            two-part ln2/256 (Cody-Waite), 2^m applied to the exponent field.
//            Out-of-range and non-finite arguments are sorted out on the integer
//            image of x, so the FP64 pipe sees 9 operations.
//  rcp_nr    hardware reciprocal approximation (rcp.approx.ftz.f64, relative
//            error ~2^-22) refined by one third-order Newton (Householder)
//            step t <- t (1 + e + e^2), e = 1 - y t, which cubes the error.
//  rsqrt_nr  hardware rsqrt approximation refined by one third-order step of
//            the binomial series y <- y (1 + e/2 + 3 e^2/8), e = 1 - s y^2.
//  erf_over_r  erf(r/r_c)/r of the screened potential from s = r^2 and 1/r:
//            with t = s/r_c^2, erf(r/r_c)/r = F(t)/r_c, F(t) = erf(sqrt t)/sqrt t,
//            an entire function of t (F(t) = (2/sqrt pi) int_0^1 exp(-t u^2) du).
//            F is tabulated as one polynomial of degree 10 per interval of
//            width 1/2 centred at k/2, k = 0..72 (Chebyshev interpolation at 11
//            nodes, rewritten in powers of t - k/2; interpolation error below
//            1e-18), evaluated by Horner; beyond t = 36.25 erf(sqrt t) rounds to
//            1 in double and the result is 1/r itself.  About 15 FP64 operations
//            against ~45 for erf and the divisions.
// The reduction constants are ln2/256 split into double hi/lo parts and
// 256/ln2, evaluated to 300 bits; the table holds 2^(j/256) rounded to double.
#pragma once

#include <cstdint>

namespace lrdmc {

constexpr int EXP_TAB = 256;
constexpr int EXP_TAB_BITS = 8;                       // EXP_TAB = 2^EXP_TAB_BITS
constexpr double EXP_INV_L = 0x1.71547652b82fep+8;    // 256 / ln 2
constexpr double EXP_L_HI = 0x1.62e42fefa39efp-9;     // ln 2 / 256, leading double
constexpr double EXP_L_LO = 0x1.abc9e3b39803fp-64;    // ln 2 / 256 - EXP_L_HI
constexpr double EXP_SHIFTER = 0x1.8p52;              // 1.5 * 2^52: rounds to an integer

// exp(x) for |x| < 700; 0 for x <= -700 (true value < 1e-304), +inf for
// x >= 700, NaN for NaN.
__device__ __forceinline__ double exp_tab(double x, const double* __restrict__ T) {
  const double t = fma(x, EXP_INV_L, EXP_SHIFTER);
  const int k = (int)__double2loint(t);                 // round(x * 256/ln2), two's complement
  const double kd = t - EXP_SHIFTER;
  double r = fma(kd, -EXP_L_HI, x);
  r = fma(kd, -EXP_L_LO, r);
  double q = fma(r, 1.0 / 24.0, 1.0 / 6.0);
  q = fma(r, q, 0.5);
  q = fma(r, q, 1.0);
  const double p = r * q;                               // exp(r) - 1
  const double tj = T[k & (EXP_TAB - 1)];
  double y = fma(tj, p, tj);
  y = __longlong_as_double(__double_as_longlong(y) + (long long)((unsigned long long)(long long)(k >> EXP_TAB_BITS) << 52));
  const unsigned hx = (unsigned)__double2hiint(x), lx = (unsigned)__double2loint(x);
  const unsigned ax = hx & 0x7fffffffu;
  const bool nan = ax > 0x7ff00000u || (ax == 0x7ff00000u && lx != 0u);
  const double big = nan ? x : ((hx >> 31) ? 0.0 : __longlong_as_double(0x7ff0000000000000ll));
  return ax >= 0x4085e000u ? big : y;                   // 0x4085e000: high word of 700.0
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
  const double t = rcp_approx(y);
  const double e = fma(-y, t, 1.0);
  return fma(t, fma(e, e, e), t);
}

// 1/sqrt(s) for s > 0 (normal range).
__device__ __forceinline__ double rsqrt_nr(double s) {
  const double y = rsqrt_approx(s);
  const double e = fma(-s, y * y, 1.0);
  return fma(y * e, fma(e, 0.375, 0.5), y);
}

// Tests on the integer image of a double, so that they issue no FP64-pipe
// instruction (the order of non-negative doubles is that of their bit
// patterns read as signed integers; a NaN has an image above +inf's).
// x > 0 and not NaN (+inf included), as (x > 0.0) evaluates:
__device__ __forceinline__ bool dpos(double x) {
  const long long b = __double_as_longlong(x);
  return b > 0 && b <= 0x7ff0000000000000ll;
}
// x != 0.0 (NaN counts as nonzero, as (x != 0.0) evaluates):
__device__ __forceinline__ bool dnonzero(double x) { return (__double_as_longlong(x) << 1) != 0; }
// x >= y for x, y >= 0 and not NaN:
__device__ __forceinline__ bool dge_nonneg(double x, double y) { return __double_as_longlong(x) >= __double_as_longlong(y); }

constexpr int ERF_INT = 73;               // intervals centred at k / 2, k = 0 .. 72
constexpr int ERF_NC = 11;                // coefficients per interval (degree 10)
constexpr double ERF_TMAX = 36.25;        // table end; erf(sqrt t) == 1 in double beyond t = 36

// erf(r / r_c) / r from s = r^2, ir = 1/r, irc2 = 1/r_c^2 and irc = 1/r_c
// (table C of ERF_INT x ERF_NC coefficients, lowest power first).
__device__ __forceinline__ double erf_over_r(double s, double ir, double irc, double irc2,
                                             const double* __restrict__ C) {
  const double t = s * irc2;
  const double y = fma(t, 2.0, EXP_SHIFTER);             // 2 t rounded to an integer in the low word
  unsigned k = (unsigned)__double2loint(y);
  k = k < (unsigned)(ERF_INT - 1) ? k : (unsigned)(ERF_INT - 1);   // in range for any t (also NaN)
  const double u = fma(y - EXP_SHIFTER, -0.5, t);          // t - k / 2
  const double* c = C + k * ERF_NC;
  double p = __ldg(c + ERF_NC - 1);
#pragma unroll
  for (int j = ERF_NC - 2; j >= 0; --j) p = fma(p, u, __ldg(c + j));
  return t < ERF_TMAX ? p * irc : ir;
}

}  // namespace lrdmc
