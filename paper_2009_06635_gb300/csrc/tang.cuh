// tang.cuh -- table-driven FP64 natural logarithm and exponential.
//
// On GB300 the FP64 pipe issues two thread-operations per clock per SM, so
// the device library's logarithm (about 28 FMA-equivalents) dominated the
// per-point FP64 work.  Both functions below follow P. T. P. Tang's
// table-driven method (logarithm: ACM TOMS 16(4), 1990, 378-400;
// exponential: ACM TOMS 15(2), 1989, 144-157), with table sizes and
// polynomial degrees of our own choosing:
//
//   ln a = e ln2 + ln F_j + log1p(u),   a = 2^e m, m in [1, 2),
//          F_j = 1 + j/256 the 1/256 step nearest to m (j = 0..256),
//          u = (m - F_j) / F_j (m - F_j exact, 1/F_j from the table),
//          |u| <= 2^-9, log1p(u) by its Taylor series to u^5
//          (truncation below 2^-54 / 6 ~ 1e-17 absolute);
//
//   e^y  = 2^M 2^(k/256) e^r,   N = round(256 y / ln2) = 256 M + k,
//          r = y - N ln2/256 with ln2/256 in two parts (Cody-Waite: the
//          fused y - N high is exact, its bits spanning less than 53
//          places for |y| < 700), |r| <= ln2/512, e^r - 1 by Taylor to r^4
//          (truncation below 4e-17 relative).
//
// ddiv: a / b by the hardware reciprocal approximation, two Newton steps and
// one product (within ~1.5 ulp; not correctly rounded), for finite nonzero
// normal b; anything else takes the exact division.
//
// Tables: {1/F_j, ln F_j} and ln(F_j / 2) for j = 0..256, 2^(k/256) for
// k = 0..255, computed on the host by the C library and staged with every
// grid (read from shared memory in the evaluation kernels, from global memory
// elsewhere).  For a in [1/2, 1) (e = -1) the sum e ln2 + ln F_j is the table
// value ln(F_j / 2) itself, so ln a for a just below 1 is not the small
// difference of two rounded logarithms (Tang's method treats the neighbourhood
// of 1 with the same aim).
//
// Domain: tlog takes a > 0 (subnormals scaled first; +inf and NaN go to the
// device library); texp takes |y| < 700 on the fast path and hands anything
// else (overflow, underflow, NaN) to the device library.
#pragma once

#include <cmath>

namespace pdfgb {

constexpr int kLogTab = 257;  // {1/F_j, ln F_j}, j = 0..256
constexpr int kExpTab = 256;  // 2^(k/256), k = 0..255

constexpr double kLn2 = 0x1.62e42fefa39efp-1;            // ln 2 rounded to double
constexpr double kInvLn2x256 = 0x1.71547652b82fep+8;     // 256 / ln 2
constexpr double kLn2d256Hi = 0x1.62e42fefa0000p-9;      // ln2/256, 36 significant bits
constexpr double kLn2d256Lo = 0x1.cf79abc9e3b3ap-48;     // ln2/256 - kLn2d256Hi
constexpr double kShifter = 0x1.8p52;                    // 1.5 * 2^52: rounds to an integer

// Host: fill the tables (logtab[2 j] = 1/F_j, logtab[2 j + 1] = ln F_j,
// loghtab[j] = ln(F_j / 2)).
void tang_tables(double *logtab, double *loghtab, double *exptab);

// The logarithm's tables: {1/F_j, ln F_j} and ln(F_j / 2).
struct LogTabs {
  const double2 *t;
  const double *h;
};

__device__ __forceinline__ double tlog(double a, LogTabs LT) {
  long long b = __double_as_longlong(a);
  int e = (int)(b >> 52) - 1023;
  if (e == -1023) {  // subnormal: bring into the normal range
    if ((b << 1) == 0) return log(a);  // zero: -inf
    b = __double_as_longlong(a * 0x1p54);
    e = (int)(b >> 52) - 1023 - 54;
  } else if (e == 1024) {
    return log(a);  // +inf, NaN
  }
  const int j = (((int)(b >> 43) & 0x1FF) + 1) >> 1;  // top 8 mantissa bits, rounded
  const double m = __longlong_as_double((b & 0x000FFFFFFFFFFFFFLL) | 0x3FF0000000000000LL);
  const double F = __longlong_as_double(0x3FF0000000000000LL + ((long long)j << 44));
  const double2 t = LT.t[j];
  const double u = (m - F) * t.x;
  double q = fma(u, 0.2, -0.25);
  q = fma(u, q, 1.0 / 3.0);
  q = fma(u, q, -0.5);
  const double p = fma(u * u, q, u);
  // a in [1/2, 1): ln(F/2) from its own table entry, so that a just below 1
  // keeps its relative precision (-ln2 + ln F would cancel)
  const double K = e == -1 ? LT.h[j] : fma((double)e, kLn2, t.y);
  return K + p;
}

__device__ __forceinline__ double ddiv(double a, double b) {
  const unsigned e = ((unsigned)(__double_as_longlong(b) >> 52)) & 0x7FFu;
  if (e < 2u || e > 2044u) return a / b;  // zero, subnormal, near over/underflow, inf, NaN
  double y;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(b));
  y = fma(y, fma(-b, y, 1.0), y);
  y = fma(y, fma(-b, y, 1.0), y);
  return a * y;
}

__device__ __forceinline__ double texp(double y, const double *ET) {
  // |y| < 700 on the fast path; the integer test keeps it off the FP64 pipe
  if ((unsigned long long)(__double_as_longlong(y) & 0x7FFFFFFFFFFFFFFFLL) >=
      (unsigned long long)__double_as_longlong(700.0))
    return exp(y);
  const double k = fma(y, kInvLn2x256, kShifter);
  const int N = __double2loint(k);
  const double kd = k - kShifter;
  double r = fma(kd, -kLn2d256Hi, y);
  r = fma(kd, -kLn2d256Lo, r);
  double q = fma(r, 1.0 / 24.0, 1.0 / 6.0);
  q = fma(r, q, 0.5);
  const double p = fma(r * r, q, r);
  const double S = ET[N & 255];
  const double v = fma(S, p, S);
  return __longlong_as_double(__double_as_longlong(v) + ((long long)(N >> 8) << 52));
}

}  // namespace pdfgb
