// ffpos.cuh -- the position of a point inside its cell, t = ln(v / v_k) / d
// (v_k the cell's first knot, d its width in ln), as a float pair, with no
// FP64 operation.
//
// On GB300 the FP64 pipe issues two operations per clock per SM; the
// table-driven FP64 logarithm and the position arithmetic were about half of
// the FP64 work of an in-grid point.  Here the logarithm of the ratio is
// reduced so that the large parts cancel exactly before any rounding
// (Tang's table method, ACM TOMS 16(4), 1990, applied to v and v_k at once):
//
//   v = 2^e m, v_k = 2^e_k m_k (m, m_k in [sqrt(1/2), sqrt(2))), F the step
//   nearest to m (1 + j/256, or half of it; j from the top mantissa bits, as
//   in tang.cuh),
//   ln(v / v_k) = (e - e_k) ln2 + (ln F - ln m_k) + log1p(u),
//   u = (m - F) / F,  |u| <= 2^-9.
//
// m - F_j is an integer multiple of 2^-52 below 2^-9, so it has at most 44
// significant bits and is split exactly into two floats (two int-to-float
// conversions of its halves).  The integer e - e_k times ln2 is exact in
// three float parts for |e - e_k| < 2^7; ln F_j and ln m_k come from tables
// as float pairs (2^-48 of their size, below 0.7); log1p(u) is u - u^2/2
// in float-float plus a float tail u^3 (1/3 - u/4 + u^2/5) (truncation below
// 2^-54 / 6).  The absolute error of the sum is a few 1e-15, about that of
// the difference of two rounded FP64 logarithms of size ~20 it replaces.
#pragma once

#include "ffmath.cuh"

namespace pdfgb {

// A double's significand is taken in [sqrt(1/2), sqrt(2)): with the top 20
// fraction bits at or above those of sqrt(2) - 1 the value is read as
// 2^(e+1) (m/2).  Then a value next to a power of two, above or below it, has
// a significand log near zero, and the log of a ratio of two close values
// cancels in small terms only.  The same test on the knots' bits (and on the
// host when their tables are made) keeps both sides consistent.
__device__ __forceinline__ bool ff_sig_high(long long b) { return ((b >> 32) & 0xFFFFF) >= 0x6A09E; }

// ln of the significand of v (a raw bit pattern, positive normal double):
// R = ln F + log1p(u), F = F_j = 1 + j/256 the step nearest to m (or F_j / 2
// for a high significand), u = (m - F_j) / F_j; e the biased exponent R goes
// with.
struct FFLnSig {
  ff2 R;
  int e;
};
__device__ __forceinline__ FFLnSig ff_ln_sig(long long bv, const float4 *LF, const float2 *LF2) {
  const bool hi = ff_sig_high(bv);
  const int j = (((int)(bv >> 43) & 0x1FF) + 1) >> 1;  // top 8 mantissa bits, rounded
  // (m - F_j) 2^52, |.| <= 2^43: dh 2^21 + dl, both halves exact in floats
  const long long d = ((bv & 0x000FFFFFFFFFFFFFLL) | 0x0010000000000000LL) - ((256LL + j) << 44);
  const int dh = (int)(d >> 21), dl = (int)(d & 0x1FFFFF);
  const ff2 dm = ff_two_sum(__fmul_rn(__int2float_rn(dh), 0x1p-31f), __fmul_rn(__int2float_rn(dl), 0x1p-52f));
  const float4 F = LF[j];
  const ff2 u = ff_mul(dm, ff2{F.x, F.y});
  // log1p(u) = u - u^2/2 + u^3 (1/3 - u/4 + u^2/5)
  const float uu = u.h;
  const float u2h = __fmul_rn(uu, uu);
  const float u2e = __fmaf_rn(uu, uu, -u2h);
  const ff2 u2 = ff_fast_sum(u2h, __fmaf_rn(2.f * uu, u.l, u2e));
  float tail = __fmaf_rn(uu, 0.2f, -0.25f);
  tail = __fmaf_rn(uu, tail, 1.f / 3.f);
  tail = __fmul_rn(__fmul_rn(u2h, uu), tail);
  ff2 l1p = ff_add(u, ff2{-0.5f * u2.h, -0.5f * u2.l});
  l1p = ff_fast_sum(l1p.h, __fadd_rn(l1p.l, tail));
  const float2 lf = hi ? LF2[j] : make_float2(F.z, F.w);
  return {ff_add(ff2{lf.x, lf.y}, l1p), (int)(bv >> 52) + (hi ? 1 : 0)};
}
// ln(v / v_k) from v's significand log and the knot's bits and ln m_k:
// (e - e_k) ln2 + (R - ln m_k), ln2 = A + B + C (A, B of 17 significant bits:
// exact products for |e - e_k| < 2^7).
__device__ __forceinline__ ff2 ff_ln_ratio(const FFLnSig &a, long long bk, float lmh, float lml) {
  const float ef = (float)(a.e - (int)(bk >> 52) - (ff_sig_high(bk) ? 1 : 0));
  ff2 s = ff_sub(a.R, ff2{lmh, lml});
  s = ff_add(s, ff_two_sum(__fmul_rn(ef, 0x1.62e4p-1f), __fmul_rn(ef, 0x1.7f7dp-20f)));
  return ff_fast_sum(s.h, __fadd_rn(s.l, __fmul_rn(ef, 0x1.cf79acp-40f)));
}

// The position of v in the cell [v_k, v_k1] of ln-width d: t = ln(v/v_k)/d
// and ts = 1 - t.  The logarithm is taken against the nearer knot (the
// positive doubles' bit patterns are nearly linear in log2, so their mean
// splits the cell near its geometric middle) and the other position is one
// minus that one, so the small position keeps its relative precision (as
// next to x = 1, where the data vanish); t = 0, ts = 1 exactly on the knot.
// kt = {ln m_k hi, lo, 1/d hi, lo}, kt1 the next knot's entry.
__device__ __forceinline__ void ff_cell_pos2(long long bv, long long bk, long long bk1, float4 kt, float4 kt1,
                                             const float4 *LF, const float2 *LF2, ff2 &t, ff2 &ts) {
  if (bv == bk) {
    t = ff2{0.f, 0.f};
    ts = ff2{1.f, 0.f};
    return;
  }
  const bool right = bv > (bk >> 1) + (bk1 >> 1);
  const FFLnSig a = ff_ln_sig(bv, LF, LF2);
  const ff2 L = ff_ln_ratio(a, right ? bk1 : bk, right ? kt1.x : kt.x, right ? kt1.y : kt.y);
  const ff2 p = ff_mul(L, right ? ff2{-kt.z, -kt.w} : ff2{kt.z, kt.w});  // the position from the nearer end
  const ff2 q = ff_sub(ff2{1.f, 0.f}, p);
  t = right ? q : p;
  ts = right ? p : q;
}
// The left-end position alone (t = 0 on the knot).
__device__ __forceinline__ ff2 ff_cell_pos(long long bv, long long bk, float4 kt, const float4 *LF,
                                           const float2 *LF2) {
  if (bv == bk) return {0.f, 0.f};
  return ff_mul(ff_ln_ratio(ff_ln_sig(bv, LF, LF2), bk, kt.x, kt.y), ff2{kt.z, kt.w});
}

}  // namespace pdfgb
