// ffsplit.cuh -- a double as a float pair on the integer and FMA pipes, for
// the adjoint's float-float paths (ff_of takes three FP64-pipe operations,
// and on GB300 the FP64 pipe issues 2 operations per clock per SM).
#pragma once

#include "ff.cuh"

namespace pdfgb {

// 0, or 2^-lim <= |v| < 2^lim: products of such weights and cotangents stay
// far inside the float exponent range, error terms included.
__device__ __forceinline__ bool ff_safe(double v, int lim) {
  const long long b = __double_as_longlong(v);
  const int e = (int)((b >> 52) & 0x7FF) - 1023;
  return (b << 1) == 0 || (e >= -lim && e < lim);
}
// A double with ff_safe(v, 50) as a float pair: the high float is the top 24
// significant bits (truncated), the low one the other 29 fraction bits as an
// integer rounded to a float and scaled by 2^(e - 52), so hi + lo is v to
// within 2^-48 of v (the integer's rounding), both of v's sign.
__device__ __forceinline__ ff2 ff_split50(double v) {
  const long long b = __double_as_longlong(v);
  if ((b << 1) == 0) return {0.f, 0.f};
  const unsigned top = (unsigned)((unsigned long long)b >> 32), sign = top & 0x80000000u;
  const int e = (int)((top >> 20) & 0x7FF) - 1023;  // |e| < 50
  const float h = __uint_as_float(sign | ((unsigned)(e + 127) << 23) | (unsigned)((b >> 29) & 0x7FFFFF));
  const float scale = __uint_as_float(sign | ((unsigned)(e - 52 + 127) << 23));
  return {h, __fmul_rn(__int2float_rn((int)(b & 0x1FFFFFFF)), scale)};
}

}  // namespace pdfgb
