// ffmath.cuh -- float-float division, logarithm and exponential on the FP32
// pipe, for the continuation rules of the FP64 evaluation.
//
// A continuation rule (the EXTRAPOLATE box of PDFFlow Fig. 1) is, per
// flavour, a quotient, a logarithm and an exponential of site values.  In
// FP64 that is ~36 operations on a pipe that issues 2 per clock per SM on
// GB300; here the same steps run on float pairs (hi + lo, ~48 significant
// bits) on the FMA pipe, 64 times wider.  What the rules need of them: the
// pair rule v = g0 exp(p ln(g1/g0)) turns an absolute error dL of the
// logarithm into a relative error |p| dL of v, and the data mass of v is
// (1 + 2|p|) times |v| at least, so the error relative to the mass stays
// below dL / 2; the low-Q^2 rule likewise (its mass grows with |rho ln rho| /
// ln 1.01 as its sensitivity to the logarithm does).  Both functions follow
// P. T. P. Tang's table-driven methods (logarithm: ACM TOMS 16(4), 1990;
// exponential: ACM TOMS 15(2), 1989) with table sizes and degrees of our own:
//
//   ln r = e ln2 - ln c_j + log1p(u),  r = 2^e m, m in [1, 2),
//          c_j = 1/F_j rounded to float, F_j = 1 + j/128 nearest to m,
//          1 + u = m c_j exactly in float-float, |u| <= 2^-8 (a little more
//          from the rounding of c_j), log1p(u) = u - u^2/2 in float-float
//          plus u^3 (1/3 - u/4 + u^2/5 - u^3/6) in float (truncation
//          below 2^-56 / 7, the float tail's rounding ~2^-49 absolute);
//
//   e^y  = 2^M 2^(k/64) (1 + expm1(r)),  N = round(64 y / ln2) = 64 M + k,
//          r = y - N ln2/64 with ln2/64 in three parts (the first N times
//          it exact), |r| <= ln2/128, expm1(r) = r + r^2/2 in float-float
//          plus r^3 (1/6 + r/24 + r^2/120 + r^3/720) in float (truncation
//          ~1e-17 relative, the tail's rounding ~2e-15 relative).
//
// Tables (host-computed in long double, each value split into float hi + lo):
// {c_j, -ln c_j} for j = 0..128 and 2^(k/64) for k = 0..63; 2 KB + 512 B.
// Domain: ff_log takes r with r.h a positive normal float; ff_exp takes
// |y.h| < 80 (the callers send anything else to the FP64 functions).
#pragma once

#include "ff.cuh"

namespace pdfgb {

constexpr int kFFLogTab = 129;  // {c_j, -ln c_j hi, -ln c_j lo, 0}, j = 0..128
constexpr int kFFExpTab = 64;   // {2^(k/64) hi, lo}, k = 0..63

// Host: fill the tables (logtab[4 j..4 j + 3] = {c_j, hi, lo, 0}, exptab[2 k..2 k + 1] = {hi, lo}).
void ff_tables(float *logtab, float *exptab);

struct FFTabs {
  const float4 *log;  // [kFFLogTab]
  const float2 *exp;  // [kFFExpTab]
};

// a + b as a normalised pair (TwoSum).
__device__ __forceinline__ ff2 ff_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bp = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bp)), __fsub_rn(b, bp));
  return {s, e};
}
// |a| >= |b| (or a == 0): a + b as a normalised pair (Fast2Sum).
__device__ __forceinline__ ff2 ff_fast_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ ff2 ff_add(ff2 a, ff2 b) {
  const ff2 s = ff_two_sum(a.h, b.h);
  return ff_fast_sum(s.h, __fadd_rn(s.l, __fadd_rn(a.l, b.l)));
}
__device__ __forceinline__ ff2 ff_sub(ff2 a, ff2 b) { return ff_add(a, ff2{-b.h, -b.l}); }
// a * f, f a float
__device__ __forceinline__ ff2 ff_mulf(ff2 a, float f) {
  const float p = __fmul_rn(a.h, f);
  const float e = __fmaf_rn(a.l, f, __fmaf_rn(a.h, f, -p));
  return ff_fast_sum(p, e);
}
// the pair as a double (exact: two float-to-double conversions on the
// integer pipe and one FP64 addition)
__device__ __forceinline__ double ff_to_d(ff2 a) { return f2d(a.h) + f2d(a.l); }

// b / a, a.h a nonzero normal float: a float quotient, then one correction
// from the remainder b - q a taken exactly (FMA).
__device__ __forceinline__ ff2 ff_div(ff2 b, ff2 a) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a.h));
  r = __fmaf_rn(r, __fmaf_rn(-a.h, r, 1.f), r);  // Newton step: ~1 ulp
  const float q = __fmul_rn(b.h, r);
  // remainder b - q a: q a.h exactly as (ph, pe), then the low parts
  const float ph = __fmul_rn(q, a.h);
  const float pe = __fmaf_rn(q, a.h, -ph);
  const float rem = __fadd_rn(__fsub_rn(__fsub_rn(b.h, ph), pe), __fmaf_rn(-q, a.l, b.l));
  return ff_fast_sum(q, __fmul_rn(rem, r));
}

// 2^e as a float, -126 <= e <= 127
__device__ __forceinline__ float ff_pow2(int e) { return __uint_as_float((unsigned)(e + 127) << 23); }

__device__ __forceinline__ ff2 ff_log(ff2 r, FFTabs T) {
  const unsigned b = __float_as_uint(r.h);
  const int e0 = (int)(b >> 23) - 127;
  const int j = (int)(((b >> 15) & 0xFFu) + 1u) >> 1;  // top 8 mantissa bits, rounded to 7
  // m = r 2^-e0 in [1, 2), exactly (a power-of-two scaling of both parts)
  const float sc = ff_pow2(-e0);
  const float mh = __fmul_rn(r.h, sc), ml = __fmul_rn(r.l, sc);
  const float4 t = T.log[j];
  // 1 + u = m c_j: the product m.h c_j exactly (ph, pe); ph - 1 is exact
  // (ph lies within a few 2^-8 of 1)
  const float ph = __fmul_rn(mh, t.x);
  const float pe = __fmaf_rn(mh, t.x, -ph);
  const ff2 u = ff_two_sum(__fsub_rn(ph, 1.f), __fmaf_rn(ml, t.x, pe));
  // log1p(u) = u - u^2/2 + u^3 (1/3 - u/4 + u^2/5 - u^3/6)
  const float uu = u.h;
  const float u2h = __fmul_rn(uu, uu);
  const float u2e = __fmaf_rn(uu, uu, -u2h);
  const ff2 u2 = ff_fast_sum(u2h, __fmaf_rn(2.f * uu, u.l, u2e));
  float tail = __fmaf_rn(uu, -1.f / 6.f, 0.2f);
  tail = __fmaf_rn(uu, tail, -0.25f);
  tail = __fmaf_rn(uu, tail, 1.f / 3.f);
  tail = __fmul_rn(__fmul_rn(u2h, uu), tail);
  ff2 l1p = ff_add(u, ff2{-0.5f * u2.h, -0.5f * u2.l});
  l1p = ff_fast_sum(l1p.h, __fadd_rn(l1p.l, tail));
  // e ln2, ln2 = A + B + C with A, B of at most 17 significant bits: e A and e B are
  // exact for |e| < 2^7, e C is rounded (~2^-24 of |e| 2^-39)
  const float ef = (float)e0;
  const ff2 eln2a = ff_two_sum(__fmul_rn(ef, 0x1.62e4p-1f), __fmul_rn(ef, 0x1.7f7dp-20f));
  const float eln2c = __fmul_rn(ef, 0x1.cf79acp-40f);
  // -ln c_j + e ln2 + log1p(u)
  ff2 s = ff_add(ff2{t.y, t.z}, eln2a);
  s = ff_add(s, l1p);
  return ff_fast_sum(s.h, __fadd_rn(s.l, eln2c));
}

__device__ __forceinline__ ff2 ff_exp(ff2 y, FFTabs T) {
  // N = round(64 y / ln2)
  const float Nf = rintf(__fmul_rn(y.h, 0x1.715476p+6f));
  const int N = __float2int_rn(Nf);
  // r = y - N ln2/64, ln2/64 = C1 + C2 + C3 (C1 of 9 significant bits, so
  // N C1 is exact for |N| < 2^13 and y.h - N C1 exact by Sterbenz; N C2 is
  // taken as its rounded product p2 and the rounding p2 - N C2)
  constexpr float C1 = 0x1.63p-7f, C2 = -0x1.bd0106p-19f, C3 = 0x1.cf79acp-46f;
  const float rh = __fmaf_rn(-Nf, C1, y.h);
  const float p2 = __fmul_rn(Nf, C2);
  const ff2 r1 = ff_two_sum(rh, -p2);
  const float c2e = __fmaf_rn(-Nf, C2, p2);  // p2 - N C2
  const ff2 r = ff_fast_sum(r1.h, __fadd_rn(r1.l, __fadd_rn(y.l, __fsub_rn(c2e, __fmul_rn(Nf, C3)))));
  // expm1(r) = r + r^2/2 + r^3 (1/6 + r/24 + r^2/120 + r^3/720)
  const float rr = r.h;
  const float r2h = __fmul_rn(rr, rr);
  const float r2e = __fmaf_rn(rr, rr, -r2h);
  const ff2 r2 = ff_fast_sum(r2h, __fmaf_rn(2.f * rr, r.l, r2e));
  float tail = __fmaf_rn(rr, 1.f / 720.f, 1.f / 120.f);
  tail = __fmaf_rn(rr, tail, 1.f / 24.f);
  tail = __fmaf_rn(rr, tail, 1.f / 6.f);
  tail = __fmul_rn(__fmul_rn(r2h, rr), tail);
  ff2 em = ff_add(r, ff2{0.5f * r2.h, 0.5f * r2.l});
  em = ff_fast_sum(em.h, __fadd_rn(em.l, tail));
  // 2^(k/64) (1 + expm1 r) = S + S expm1(r), then the power of two
  const float2 S = T.exp[N & 63];
  const ff2 Sem = ff_mul(ff2{S.x, S.y}, em);
  ff2 v = ff_add(ff2{S.x, S.y}, Sem);
  const int M = N >> 6;  // floor(N / 64)
  // 2^M in two steps so that M down to -252 stays normal on the way
  const float s1 = ff_pow2(M / 2), s2 = ff_pow2(M - M / 2);
  return {__fmul_rn(__fmul_rn(v.h, s1), s2), __fmul_rn(__fmul_rn(v.l, s1), s2)};
}

}  // namespace pdfgb
