// xf64.cu -- FP64 evaluation of x f(x, Q^2): points (all flavours or a
// column range), Monte Carlo events, member sets; alpha_s(Q^2) optionally
// in the same pass.
//
// One warp owns a tile of 32 points (16 events).  Phase 1 (lane = point):
// load (coalesced), classify and search on bit patterns, ln x and ln Q^2 by
// the table-driven logarithm (tang.cuh), alpha_s.  Points inside the grid
// (and invalid ones) take a slot of the warp's record.  Points that need a
// continuation rule (x < x0 or Q^2 outside the grid) are pushed onto the
// warp's queue in shared memory instead and evaluated 32 at a time once the
// queue holds a full tile (the rest at the end): their logarithms and
// exponentials then run in full warps, not in the few lanes a mixed tile
// would leave them.  Member sets skip the queue (a point's hundreds of
// member items fill the warp anyway).
// Phase 2 (lane = item (point, column); consecutive items are consecutive
// outputs, so stores coalesce): in-grid points contract the cell's 16
// float-float control points with float-float Bernstein weights on the FP32
// pipe (GB300 issues FP32 at 64x its FP64 rate; the result is good to about
// 2^-46 of the data scale); exact knot hits use FP64.  Continuation points
// evaluate their sites and rules in float-float too (ffmath.cuh: quotient,
// logarithm and exponential on the FP32 pipe; FP64 only for the final sum and
// for exponents beyond the float range), on grids whose control points are
// in float-float range; other grids keep the FP64 rules.  The continuation
// classes share one copy of the pair rule, so lanes of different classes
// reconverge before its logarithm and exponential.
#include <cmath>

#include "mc.cuh"
#include "ff.cuh"
#include "ffmath.cuh"
#include "sites.cuh"

namespace pdfgb {

namespace {

constexpr int kWarps = 8;
constexpr int kThreads = 32 * kWarps;
constexpr unsigned kFull = 0xffffffffu;

// Per-warp record of the points of one tile, by class-sorted slot.  Each
// slot owns one 144-byte row of weights: for C_INF the 16 float-float
// products Bx[k] Bq[l] (hi, lo) at [l*4 + k], for C_IN the same products in
// FP64, otherwise Bx0 | Bx1 | Bq0 | Bq1 in FP64.  Rows are padded from 128
// to 144 bytes so that the few slots one load instruction touches fall in
// different banks, and stay 16-byte aligned for paired loads.
struct alignas(16) Rec64 {
  int cls[32], xc0[32], xc1[32], qc0[32], qc1[32];
  long long ob[32];  // output offset of the point's first column
  double W[32][18];
  double px[32], pq[32], lr[32];
};
// Continuation points waiting for a full tile, one queue per class (at most
// 31 + 32 each), as point indices (MODE_MC: event index times 2 plus the side);
// a drain reads the coordinates again.  Full tiles of one class run one code
// path; only the leftovers at the end mix classes.
constexpr int kFar = C_LOWX_LOWQ - C_LOWX + 1;  // continuation classes
struct alignas(16) Queue64 {
  unsigned idx[kFar][64];
};

// sum_m w_m b_m with w from the record and b from the float-float control
// points (c: the item's first pair of control points; pairs nf float4
// apart), as two chains run side by side in packed f32x2 operations (GB300
// issues one instruction for both halves): chain 0 takes the even control
// points m = 2 m2, chain 1 the odd ones.  Both the record row and the control
// points hold a pair as {hi_even, hi_odd, lo_even, lo_odd}, so the halves of
// each operand sit in one register pair.  Each chain adds exact products by
// TwoSum and gathers the cross terms and rounding errors in a second float;
// the chains are merged by one more TwoSum at the end.
__device__ __forceinline__ double dot_ff16(const float4 *c, int nf, const float4 *w) {
  float2 sh = make_float2(0.f, 0.f), sl = make_float2(0.f, 0.f);
#pragma unroll
  for (int m2 = 0; m2 < 8; m2++) {
    const float4 ww = w[m2];
    const float4 bb = __ldg(c + (size_t)m2 * nf);
    const float2 wh = make_float2(ww.x, ww.y), wl = make_float2(ww.z, ww.w);
    const float2 bh = make_float2(bb.x, bb.y), bl = make_float2(bb.z, bb.w);
    const float2 ph = __fmul2_rn(wh, bh);
    float2 pe = __ffma2_rn(wh, bh, neg2(ph));
    pe = __ffma2_rn(wh, bl, __ffma2_rn(wl, bh, pe));
    const float2 t = __fadd2_rn(sh, ph);
    const float2 bp = __fadd2_rn(t, neg2(sh));
    const float2 err = __fadd2_rn(__fadd2_rn(sh, neg2(__fadd2_rn(t, neg2(bp)))), __fadd2_rn(ph, neg2(bp)));
    sh = t;
    sl = __fadd2_rn(sl, __fadd2_rn(err, pe));
  }
  const float s = __fadd_rn(sh.x, sh.y);
  const float bp = __fsub_rn(s, sh.x);
  const float e = __fadd_rn(__fsub_rn(sh.x, __fsub_rn(s, bp)), __fsub_rn(sh.y, bp));
  return f2d(s) + f2d(__fadd_rn(__fadd_rn(sl.x, sl.y), e));
}

// ---- FP64 site evaluation ---------------------------------------------------
__device__ __forceinline__ double dot_w16(const double *c, const Rec64 &R, int p) {
  const double2 *q = reinterpret_cast<const double2 *>(c);
  double2 v = __ldg(q);
  double acc = R.W[p][0] * v.x;
  acc = fma(R.W[p][1], v.y, acc);
#pragma unroll
  for (int m = 1; m < 8; m++) {
    v = __ldg(q + m);
    acc = fma(R.W[p][2 * m], v.x, acc);
    acc = fma(R.W[p][2 * m + 1], v.y, acc);
  }
  return acc;
}
// site with t general, u general: sum_l Bq[l] sum_k Bx[k] b[l][k]
__device__ __forceinline__ double site_tu(const double *c, const Rec64 &R, int p, int a, int b) {
  double f = 0.0;
#pragma unroll
  for (int l = 0; l < 4; l++) {
    const double2 *q = reinterpret_cast<const double2 *>(c + 4 * l);
    double2 v0 = __ldg(q), v1 = __ldg(q + 1);
    double r = R.W[p][4 * a] * v0.x;
    r = fma(R.W[p][4 * a + 1], v0.y, r);
    r = fma(R.W[p][4 * a + 2], v1.x, r);
    r = fma(R.W[p][4 * a + 3], v1.y, r);
    f = l == 0 ? R.W[p][8 + 4 * b] * r : fma(R.W[p][8 + 4 * b + l], r, f);
  }
  return f;
}
// site on an x knot (t = 0): sum_l Bq[l] b[l][0]
__device__ __forceinline__ double site_u(const double *c, const Rec64 &R, int p, int b) {
  double f = R.W[p][8 + 4 * b] * __ldg(c);
  f = fma(R.W[p][8 + 4 * b + 1], __ldg(c + 4), f);
  f = fma(R.W[p][8 + 4 * b + 2], __ldg(c + 8), f);
  return fma(R.W[p][8 + 4 * b + 3], __ldg(c + 12), f);
}
// site on a Q knot (u = 0): sum_k Bx[k] b[0][k]
__device__ __forceinline__ double site_t(const double *c, const Rec64 &R, int p, int a) {
  const double2 *q = reinterpret_cast<const double2 *>(c);
  double2 v0 = __ldg(q), v1 = __ldg(q + 1);
  double f = R.W[p][4 * a] * v0.x;
  f = fma(R.W[p][4 * a + 1], v0.y, f);
  f = fma(R.W[p][4 * a + 2], v1.x, f);
  return fma(R.W[p][4 * a + 3], v1.y, f);
}

// ---- float-float continuation ------------------------------------------------
// A continuation point's record row holds its Bernstein weights as float
// pairs, W2[0..3] Bx0, [4..7] Bx1, [8..11] Bq0, [12..15] Bq1, and px, pq, lr
// as float pairs in the same 8-byte slots.  Sites contract the float-float
// control points (coefff: pair m2 of control points m = 2 m2, 2 m2 + 1 of a
// flavour as one float4 {hi_m, hi_m+1, lo_m, lo_m+1} with m = 2 m2;
// control point m = 4 l + k).
__device__ __forceinline__ ff2 ffv(const double &d) {
  const float2 v = reinterpret_cast<const float2 &>(d);
  return {v.x, v.y};
}
__device__ __forceinline__ ff2 ffw(const float2 &w) { return {w.x, w.y}; }
__device__ __forceinline__ ff2 ff_norm(float sh, float sl) { return ff_two_sum(sh, sl); }
// on an x knot (t = 0): sum_l Bq[l] b[l][0]
__device__ __forceinline__ ff2 ffsite_u(const float4 *c, int nfp, const float2 *bq) {
  float sh = 0.f, sl = 0.f;
#pragma unroll
  for (int l = 0; l < 4; l++) {
    const float4 v = __ldg(c + (size_t)(2 * l) * nfp);  // control point m = 4 l: the pair's even one
    ff_acc(sh, sl, ffw(bq[l]), v.x, v.z);
  }
  return ff_norm(sh, sl);
}
// on a Q knot (u = 0): sum_k Bx[k] b[0][k]
__device__ __forceinline__ ff2 ffsite_t(const float4 *c, int nfp, const float2 *bx) {
  const float4 v0 = __ldg(c), v1 = __ldg(c + nfp);
  float sh = 0.f, sl = 0.f;
  ff_acc(sh, sl, ffw(bx[0]), v0.x, v0.z);
  ff_acc(sh, sl, ffw(bx[1]), v0.y, v0.w);
  ff_acc(sh, sl, ffw(bx[2]), v1.x, v1.z);
  ff_acc(sh, sl, ffw(bx[3]), v1.y, v1.w);
  return ff_norm(sh, sl);
}
// general: sum_l Bq[l] sum_k Bx[k] b[l][k]
__device__ __forceinline__ ff2 ffsite_tu(const float4 *c, int nfp, const float2 *bx, const float2 *bq) {
  float sh = 0.f, sl = 0.f;
#pragma unroll
  for (int l = 0; l < 4; l++) {
    const ff2 r = ffsite_t(c + (size_t)(2 * l) * nfp, nfp, bx);
    ff_acc(sh, sl, ffw(bq[l]), r.h, r.l);
  }
  return ff_norm(sh, sl);
}
__device__ __forceinline__ ff2 ffknot(const float4 *c) {
  const float4 v = __ldg(c);
  return {v.x, v.z};
}

// A rule's result: a float pair, or (out of the pairs' range) a double.
struct FFRes {
  ff2 v;
  double d;
  bool dbl;
};
__device__ __forceinline__ ff2 res_ff(const FFRes &r) { return r.dbl ? ff_of(r.d) : r.v; }
__device__ __forceinline__ double res_d(const FFRes &r) { return r.dbl ? r.d : ff_to_d(r.v); }

// The FP64 steps the float-pair rules fall back on (out of line: they are
// rare, and inlined they would take registers from the common path).
__device__ __noinline__ double pair_rule_fp64(double g0, double g1, double p) { return g0 * exp(p * log(g1 / g0)); }
__device__ __noinline__ double lowq_rule_fp64(double f0, double f1, double rho, double lr, double iln101, bool pos) {
  const double g = pos ? log(f1 / f0) * iln101 : 1.0;
  return f0 * exp(((g * rho + 1.0) - rho) * lr);
}

// The pair rule: g0 (g1/g0)^p if both are > 0, else g0 + (g1 - g0) p.
// Float pairs keep ~48 bits only while their low part is a normal float:
// a quotient outside [2^-100, 2^100], an exponent beyond +-64 or a result
// below 2^-100 in magnitude is taken again in FP64.
constexpr float kFFLo = 0x1p-100f, kFFHi = 0x1p100f;
__device__ __forceinline__ bool ff_ok(ff2 v) { return fabsf(v.h) >= kFFLo && fabsf(v.h) < kFFHi; }
__device__ __forceinline__ FFRes ff_pair_rule(ff2 g0, ff2 g1, ff2 p, FFTabs FT) {
  if (g0.h > 0.f && g1.h > 0.f) {
    const ff2 r = ff_div(g1, g0);
    if (ff_ok(r)) {
      const ff2 y = ff_mul(p, ff_log(r, FT));
      if (fabsf(y.h) < 64.f) {
        const ff2 v = ff_mul(g0, ff_exp(y, FT));
        if (ff_ok(v)) return {v, 0.0, false};
      }
    }
    return {{0.f, 0.f}, pair_rule_fp64(ff_to_d(g0), ff_to_d(g1), ff_to_d(p)), true};
  }
  return {ff_add(g0, ff_mul(ff_sub(g1, g0), p)), 0.0, false};
}
// The low-Q^2 rule: gamma = ln(f1/f0) / ln 1.01 if both are > 0, else 1;
// f0 rho^(gamma rho + 1 - rho) as f0 exp((gamma rho + 1 - rho) ln rho).
__device__ __forceinline__ FFRes ff_lowq_rule(ff2 f0, ff2 f1, ff2 rho, ff2 lr, ff2 iln101, FFTabs FT) {
  const bool pos = f0.h > 0.f && f1.h > 0.f;
  ff2 gam = {1.f, 0.f};
  bool fp64 = false;
  if (pos) {
    const ff2 r = ff_div(f1, f0);
    if (ff_ok(r)) gam = ff_mul(ff_log(r, FT), iln101);
    else fp64 = true;
  }
  if (!fp64) {
    const ff2 ex = ff_sub(ff_add(ff_mul(gam, rho), ff2{1.f, 0.f}), rho);
    const ff2 y = ff_mul(ex, lr);
    if (fabsf(y.h) < 64.f) {
      const ff2 v = ff_mul(f0, ff_exp(y, FT));
      if (ff_ok(v) || f0.h == 0.f) return {v, 0.0, false};
    }
  }
  return {{0.f, 0.f}, lowq_rule_fp64(ff_to_d(f0), ff_to_d(f1), ff_to_d(rho), ff_to_d(lr), ff_to_d(iln101), pos), true};
}

// A continuation item in float-float (the grid's control points are in range).
__device__ __forceinline__ double eval_far_ff(const GridView &g, const Rec64 &R, int p, int col, int m,
                                              FFTabs FT) {
  const float4 *cb = reinterpret_cast<const float4 *>(g.coefff + (size_t)m * g.mstride_ff) + col;
  const size_t cstride = (size_t)8 * g.nfp;  // float4 per cell
  const int nfp = g.nfp;
  auto C = [&](int a, int b) {
    const int xc = a ? R.xc1[p] : R.xc0[p];
    const int qc = b ? R.qc1[p] : R.qc0[p];
    return cb + ((size_t)qc * g.nx + xc) * cstride;
  };
  const float2 *W2 = reinterpret_cast<const float2 *>(R.W[p]);
  const ff2 il = ff2{g.iln101_ffh, g.iln101_ffl};
  ff2 a, b, prm = ffv(R.px[p]);
  switch (R.cls[p]) {
    case C_LOWX:  // sites (x0, Q^2), (x1, Q^2): t = 0
      a = ffsite_u(C(0, 0), nfp, W2 + 8);
      b = ffsite_u(C(1, 0), nfp, W2 + 8);
      break;
    case C_HIGHQ:  // sites (x, Q2max), (x, knot below): u = 0
      a = ffsite_t(C(0, 0), nfp, W2);
      b = ffsite_t(C(0, 1), nfp, W2);
      prm = ffv(R.pq[p]);
      break;
    case C_LOWQ:  // sites (x, Q2min): u = 0; (x, 1.01 Q2min): general
      return res_d(ff_lowq_rule(ffsite_t(C(0, 0), nfp, W2), ffsite_tu(C(0, 1), nfp, W2, W2 + 12), ffv(R.pq[p]),
                                ffv(R.lr[p]), il, FT));
    case C_LOWX_HIGHQ:  // all four sites are knots
      a = res_ff(ff_pair_rule(ffknot(C(0, 0)), ffknot(C(0, 1)), ffv(R.pq[p]), FT));
      b = res_ff(ff_pair_rule(ffknot(C(1, 0)), ffknot(C(1, 1)), ffv(R.pq[p]), FT));
      break;
    default:  // C_LOWX_LOWQ
      a = res_ff(ff_lowq_rule(ffknot(C(0, 0)), ffsite_u(C(0, 1), nfp, W2 + 12), ffv(R.pq[p]), ffv(R.lr[p]), il, FT));
      b = res_ff(ff_lowq_rule(ffknot(C(1, 0)), ffsite_u(C(1, 1), nfp, W2 + 12), ffv(R.pq[p]), ffv(R.lr[p]), il, FT));
      break;
  }
  return res_d(ff_pair_rule(a, b, prm, FT));
}

// One item: column col of the point in slot p, of member m.
// RCP: the low-Q^2 rule multiplies by 1 / ln 1.01 (the Monte Carlo kernel,
// where a fifth of the events take it; the other kernels keep the division,
// which left their register allocation as measured fastest).
// FAR: the continuation classes may occur (the near launch has none, and
// leaves their code out).
template <bool RCP, bool FAR>
__device__ __forceinline__ double eval_item64(const GridView &g, const Rec64 &R, int p, int col, int m,
                                              LogTabs LT, const double *ET, FFTabs FT) {
  const double *cb = g.coef + (size_t)m * g.mstride + (size_t)col * 16;
  const size_t stride = (size_t)g.nf * 16;
  auto C = [&](int a, int b) {
    int xc = a ? R.xc1[p] : R.xc0[p];
    int qc = b ? R.qc1[p] : R.qc0[p];
    return cb + ((size_t)qc * g.nx + xc) * stride;
  };
  const int cls = R.cls[p];
  if (cls == C_INF)
    return dot_ff16(reinterpret_cast<const float4 *>(g.coefff + (size_t)m * g.mstride_ff +
                                                     ((size_t)R.qc0[p] * g.nx + R.xc0[p]) * 16 * g.nfp) + col,
                    g.nfp, reinterpret_cast<const float4 *>(R.W[p]));
  if (cls == C_IN) return dot_w16(C(0, 0), R, p);
  if (cls == C_INVALID) return NAN;
  if constexpr (!FAR) return NAN;
  if (g.ff) return eval_far_ff(g, R, p, col, m, FT);
  // continuation: the two values the final rule combines, then one shared rule
  double a, b, prm = R.px[p];
  bool lowq = false;
  switch (cls) {
    case C_LOWX:  // sites (x0, Q^2), (x1, Q^2): t = 0
      a = site_u(C(0, 0), R, p, 0);
      b = site_u(C(1, 0), R, p, 0);
      break;
    case C_HIGHQ:  // sites (x, Q2max), (x, knot below): u = 0
      a = site_t(C(0, 0), R, p, 0);
      b = site_t(C(0, 1), R, p, 0);
      prm = R.pq[p];
      break;
    case C_LOWQ:  // sites (x, Q2min): u = 0; (x, 1.01 Q2min): general
      a = site_t(C(0, 0), R, p, 0);
      b = site_tu(C(0, 1), R, p, 0, 1);
      lowq = true;
      break;
    case C_LOWX_HIGHQ:  // all four sites are knots
      a = pair_rule(__ldg(C(0, 0)), __ldg(C(0, 1)), R.pq[p], LT, ET);
      b = pair_rule(__ldg(C(1, 0)), __ldg(C(1, 1)), R.pq[p], LT, ET);
      break;
    default:  // C_LOWX_LOWQ
      if constexpr (RCP) {
        a = lowq_rule_r(__ldg(C(0, 0)), site_u(C(0, 1), R, p, 1), R.pq[p], R.lr[p], g.iln101, LT, ET);
        b = lowq_rule_r(__ldg(C(1, 0)), site_u(C(1, 1), R, p, 1), R.pq[p], R.lr[p], g.iln101, LT, ET);
      } else {
        a = lowq_rule(__ldg(C(0, 0)), site_u(C(0, 1), R, p, 1), R.pq[p], R.lr[p], g.ln101, LT, ET);
        b = lowq_rule(__ldg(C(1, 0)), site_u(C(1, 1), R, p, 1), R.pq[p], R.lr[p], g.ln101, LT, ET);
      }
      break;
  }
  if constexpr (RCP) {
    if (lowq) return lowq_rule_r(a, b, R.pq[p], R.lr[p], g.iln101, LT, ET);
  } else {
    if (lowq) return lowq_rule(a, b, R.pq[p], R.lr[p], g.ln101, LT, ET);
  }
  return pair_rule(a, b, prm, LT, ET);
}

// ---- near launch on float-float grids: positions without FP64 -------------
// An in-grid point's cell positions t, u (and 1 - t, 1 - u) as float pairs
// (ffpos.cuh); points of the other classes are only classified here.
struct NearFF {
  int cls, xc0, qc0;
  ff2 t, ts, u, us;
};
__device__ __forceinline__ NearFF near_sites_ff(const GridView &g, const long long *xkeys,
                                                const long long *qkeys, const float4 *LF, const float2 *LF2,
                                                double x, double q2, const PosTabs &T) {
  NearFF r;
  r.xc0 = r.qc0 = 0;
  r.t = r.u = ff2{0.f, 0.f};
  r.ts = r.us = ff2{1.f, 0.f};
  const long long kx = __double_as_longlong(x), kq = __double_as_longlong(q2);
  if (!(kq > 0 && kq < 0x7FF0000000000000LL && kx > 0 && kx <= __double_as_longlong(g.xlast))) {
    r.cls = C_INVALID;
    return r;
  }
  const bool lowx = kx < __double_as_longlong(g.x0);
  const bool lowq = kq < __double_as_longlong(g.q2min), highq = kq > __double_as_longlong(g.q2max);
  if (lowx || lowq || highq) {
    r.cls = lowx ? (highq ? C_LOWX_HIGHQ : lowq ? C_LOWX_LOWQ : C_LOWX) : (highq ? C_HIGHQ : C_LOWQ);
    return r;
  }
  const int i = search_cell(xkeys, g.nx, g.xstep, kx);
  const int j = search_cell(qkeys, g.nrows, g.qstep, kq);
  r.xc0 = i;
  r.qc0 = T.row_qc[j];
  // (an exact hit on the last knot, or the top row, is the knot case: no next knot is read)
  const bool xk1 = kx != xkeys[i], qk1 = kq != qkeys[j];
  ff_cell_pos2(kx, xkeys[i], xk1 ? xkeys[i + 1] : 0, T.xpos[i], xk1 ? T.xpos[i + 1] : make_float4(0.f, 0.f, 0.f, 0.f),
               LF, LF2, r.t, r.ts);
  ff_cell_pos2(kq, qkeys[j], qk1 ? qkeys[j + 1] : 0, T.qpos[j], qk1 ? T.qpos[j + 1] : make_float4(0.f, 0.f, 0.f, 0.f),
               LF, LF2, r.u, r.us);
  // an exact knot hit (t = u = 0) keeps the FP64 contraction, so knot values come back exactly
  r.cls = (r.t.h == 0.f && r.u.h == 0.f) ? C_IN : C_INF;
  return r;
}
// Bernstein basis from a float-pair position and its complement.
__device__ __forceinline__ void ff_bernstein2(ff2 tf, ff2 sf, ff2 *B) {
  const ff2 three = {3.f, 0.f};
  const ff2 t2 = ff_mul(tf, tf), s2 = ff_mul(sf, sf);
  B[0] = ff_mul(s2, sf);
  B[1] = ff_mul(three, ff_mul(tf, s2));
  B[2] = ff_mul(three, ff_mul(t2, sf));
  B[3] = ff_mul(t2, tf);
}
__device__ __forceinline__ void store_point_ff(Rec64 &R, int slot, const NearFF &ps, long long ob) {
  R.cls[slot] = ps.cls;
  R.xc0[slot] = ps.xc0; R.xc1[slot] = 0; R.qc0[slot] = ps.qc0; R.qc1[slot] = 0;
  R.ob[slot] = ob;
  if (ps.cls == C_INF) {
    ff2 bx[4], bq[4];
    ff_bernstein2(ps.t, ps.ts, bx);
    ff_bernstein2(ps.u, ps.us, bq);
    float4 *row = reinterpret_cast<float4 *>(R.W[slot]);
#pragma unroll
    for (int l = 0; l < 4; l++)
#pragma unroll
      for (int k = 0; k < 4; k += 2) {
        const ff2 w0 = ff_mul(bx[k], bq[l]), w1 = ff_mul(bx[k + 1], bq[l]);
        row[(l * 4 + k) >> 1] = make_float4(w0.h, w1.h, w0.l, w1.l);
      }
  } else if (ps.cls == C_IN) {  // an exact knot: the weight of control point 0 alone
#pragma unroll
    for (int m = 0; m < 16; m++) R.W[slot][m] = m == 0 ? 1.0 : 0.0;
  }
}

// ---- continued points on float-float grids: sites without FP64 -------------
// The sites and rule parameters of a point outside the grid (as sites() and
// store_point give them) from ffpos.cuh: the in-grid coordinate's position,
// p_x = ln(x/x0)/d0 below x0, p_q = -ln(Q^2/Q2max)/d_top above Q2max, and
// below Q2min rho = Q^2/Q2min (one FP64 product) with ln rho.  The other
// sites sit on knots (t = 0) except the low-Q^2 one at 1.01 Q2min.
struct FarFF {
  int cls, xc0, xc1, qc0, qc1;
  bool q101;  // the second Q site is 1.01 Q2min (else a knot)
  ff2 t0, ts0, u0, us0, px, pq, lr;
};
__device__ __forceinline__ FarFF far_sites_ff(const GridView &g, const long long *xkeys, const long long *qkeys,
                                              const float4 *LF, const float2 *LF2, double x, double q2,
                                              const PosTabs &T) {
  FarFF r;
  r.xc0 = r.xc1 = r.qc0 = r.qc1 = 0;
  r.q101 = false;
  r.t0 = r.u0 = r.px = r.pq = r.lr = ff2{0.f, 0.f};
  r.ts0 = r.us0 = ff2{1.f, 0.f};
  const long long kx = __double_as_longlong(x), kq = __double_as_longlong(q2);
  if (!(kq > 0 && kq < 0x7FF0000000000000LL && kx > 0 && kx <= __double_as_longlong(g.xlast))) {
    r.cls = C_INVALID;
    return r;
  }
  const bool lowx = kx < __double_as_longlong(g.x0);
  const bool lowq = kq < __double_as_longlong(g.q2min), highq = kq > __double_as_longlong(g.q2max);
  if (!lowx) {
    const int i = search_cell(xkeys, g.nx, g.xstep, kx);
    r.xc0 = i;
    const bool k1 = kx != xkeys[i];
    ff_cell_pos2(kx, xkeys[i], k1 ? xkeys[i + 1] : 0, T.xpos[i], k1 ? T.xpos[i + 1] : make_float4(0.f, 0.f, 0.f, 0.f),
                 LF, LF2, r.t0, r.ts0);
  } else {
    r.xc1 = 1;
    const float4 k0 = T.xpos[0];
    r.px = ff_mul(ff_ln_ratio(ff_ln_sig(kx, LF, LF2), xkeys[0], k0.x, k0.y), ff2{k0.z, k0.w});
  }
  if (!lowq && !highq) {
    const int j = search_cell(qkeys, g.nrows, g.qstep, kq);
    r.qc0 = T.row_qc[j];
    const bool k1 = kq != qkeys[j];
    ff_cell_pos2(kq, qkeys[j], k1 ? qkeys[j + 1] : 0, T.qpos[j], k1 ? T.qpos[j + 1] : make_float4(0.f, 0.f, 0.f, 0.f),
                 LF, LF2, r.u0, r.us0);
  } else if (highq) {
    r.qc0 = g.nqc;
    r.qc1 = g.top_qc;
    const float4 kt = T.qpos[g.nrows - 1], kc = T.qpos[g.nrows - 2];  // Q2max; its cell's width
    r.pq = ff_mul(ff_ln_ratio(ff_ln_sig(kq, LF, LF2), qkeys[g.nrows - 1], kt.x, kt.y), ff2{-kc.z, -kc.w});
  } else {
    r.qc1 = g.q101_qc;
    r.q101 = true;
    r.pq = ff_of(q2 * g.inv_q2min);
    const float4 k0 = T.qpos[0];
    r.lr = ff_ln_ratio(ff_ln_sig(kq, LF, LF2), qkeys[0], k0.x, k0.y);
  }
  r.cls = lowx ? (highq ? C_LOWX_HIGHQ : lowq ? C_LOWX_LOWQ : C_LOWX) : (highq ? C_HIGHQ : lowq ? C_LOWQ : C_IN);
  return r;
}
__device__ __forceinline__ void store_point_far_ff(Rec64 &R, int slot, const FarFF &ps, long long ob,
                                                   const GridView &g) {
  R.cls[slot] = ps.cls;
  R.xc0[slot] = ps.xc0; R.xc1[slot] = ps.xc1; R.qc0[slot] = ps.qc0; R.qc1[slot] = ps.qc1;
  R.ob[slot] = ob;
  if (ps.cls == C_INVALID) return;
  reinterpret_cast<float2 &>(R.px[slot]) = make_float2(ps.px.h, ps.px.l);
  reinterpret_cast<float2 &>(R.pq[slot]) = make_float2(ps.pq.h, ps.pq.l);
  reinterpret_cast<float2 &>(R.lr[slot]) = make_float2(ps.lr.h, ps.lr.l);
  float2 *W2 = reinterpret_cast<float2 *>(R.W[slot]);
  ff2 B[4];
  ff_bernstein2(ps.t0, ps.ts0, B);
#pragma unroll
  for (int k = 0; k < 4; k++) W2[k] = make_float2(B[k].h, B[k].l);
#pragma unroll
  for (int k = 0; k < 4; k++) W2[4 + k] = make_float2(k == 0 ? 1.f : 0.f, 0.f);  // on a knot: t = 0
  ff_bernstein2(ps.u0, ps.us0, B);
#pragma unroll
  for (int k = 0; k < 4; k++) W2[8 + k] = make_float2(B[k].h, B[k].l);
  if (ps.q101) {
    ff_bernstein2(ff2{g.q101ff[0], g.q101ff[1]}, ff2{g.q101ff[2], g.q101ff[3]}, B);
#pragma unroll
    for (int k = 0; k < 4; k++) W2[12 + k] = make_float2(B[k].h, B[k].l);
  } else {
#pragma unroll
    for (int k = 0; k < 4; k++) W2[12 + k] = make_float2(k == 0 ? 1.f : 0.f, 0.f);
  }
}

// Bernstein weights of a point's sites into its record slot (float-float
// for continuation points when ff is set).
__device__ __forceinline__ void store_point(Rec64 &R, int slot, const PointSites<double> &ps, long long ob,
                                            int ff) {
  R.cls[slot] = ps.cls;
  R.xc0[slot] = ps.xc0; R.xc1[slot] = ps.xc1; R.qc0[slot] = ps.qc0; R.qc1[slot] = ps.qc1;
  R.ob[slot] = ob;
  R.px[slot] = ps.px; R.pq[slot] = ps.pq; R.lr[slot] = ps.lr;
  if (ps.cls == C_INVALID) return;
  if (ff && ps.cls >= C_LOWX && ps.cls <= C_LOWX_LOWQ) {
    auto put = [](double &slot_, double v) {
      const ff2 f = ff_of(v);
      reinterpret_cast<float2 &>(slot_) = make_float2(f.h, f.l);
    };
    put(R.px[slot], ps.px);
    put(R.pq[slot], ps.pq);
    put(R.lr[slot], ps.lr);
    ff2 B[4];
    float2 *W2 = reinterpret_cast<float2 *>(R.W[slot]);
    ff_bernstein(ps.t0, ps.ts0, B);
#pragma unroll
    for (int k = 0; k < 4; k++) W2[k] = make_float2(B[k].h, B[k].l);
    ff_bernstein(ps.t1, 1.0 - ps.t1, B);
#pragma unroll
    for (int k = 0; k < 4; k++) W2[4 + k] = make_float2(B[k].h, B[k].l);
    ff_bernstein(ps.u0, ps.us0, B);
#pragma unroll
    for (int k = 0; k < 4; k++) W2[8 + k] = make_float2(B[k].h, B[k].l);
    ff_bernstein(ps.u1, 1.0 - ps.u1, B);
#pragma unroll
    for (int k = 0; k < 4; k++) W2[12 + k] = make_float2(B[k].h, B[k].l);
    return;
  }
  if (ps.cls == C_INF) {
    ff2 bx[4], bq[4];
    ff_bernstein(ps.t0, ps.ts0, bx);
    ff_bernstein(ps.u0, ps.us0, bq);
    // pairs of products m = 2 m2, 2 m2 + 1 as {hi, hi, lo, lo} (dot_ff16)
    float4 *row = reinterpret_cast<float4 *>(R.W[slot]);
#pragma unroll
    for (int l = 0; l < 4; l++)
#pragma unroll
      for (int k = 0; k < 4; k += 2) {
        const ff2 w0 = ff_mul(bx[k], bq[l]), w1 = ff_mul(bx[k + 1], bq[l]);
        row[(l * 4 + k) >> 1] = make_float4(w0.h, w1.h, w0.l, w1.l);
      }
    return;
  }
  double bx0[4], bq0[4];
  bernstein<double>(ps.t0, ps.ts0, bx0);
  bernstein<double>(ps.u0, ps.us0, bq0);
  if (ps.cls == C_IN) {
#pragma unroll
    for (int l = 0; l < 4; l++)
#pragma unroll
      for (int k = 0; k < 4; k++) R.W[slot][l * 4 + k] = bx0[k] * bq0[l];
    return;
  }
  double bx1[4], bq1[4];
  bernstein<double>(ps.t1, 1.0 - ps.t1, bx1);
  bernstein<double>(ps.u1, 1.0 - ps.u1, bq1);
#pragma unroll
  for (int k = 0; k < 4; k++) {
    R.W[slot][k] = bx0[k];
    R.W[slot][4 + k] = bx1[k];
    R.W[slot][8 + k] = bq0[k];
    R.W[slot][12 + k] = bq1[k];
  }
}

// Phase 2 over the first np slots: items (slot, column) in order, lane-strided.
template <bool RCP, bool FAR = true>
__device__ __forceinline__ void items64(const GridView &g, const Rec64 &R, int np, int nc, int cbase,
                                        int m, long long mo, double *__restrict__ out, LogTabs LT,
                                        const double *ET, FFTabs FT, int lane) {
  const int nitems = np * nc;
  int p = lane / nc, c = lane - (lane / nc) * nc;
  const int dp = 32 / nc, dc = 32 - dp * nc;
  for (int k = lane; k < nitems; k += 32) {
    out[mo + R.ob[p] + c] = eval_item64<RCP, FAR>(g, R, p, cbase + c, m, LT, ET, FT);
    c += dc;
    p += dp;
    if (c >= nc) { c -= nc; p++; }
  }
}

__device__ __forceinline__ bool is_far(int cls) { return cls >= C_LOWX && cls <= C_LOWX_LOWQ; }

// Counting sort of the lanes whose key is one of the classes Cs (in that
// order), by ballots; returns the number of slots used.
template <int... Cs>
__device__ __forceinline__ int sort_slots(int key, int lane, int &slot) {
  const unsigned lt = (1u << lane) - 1u;
  int base = 0;
  auto one = [&](int c) {
    const unsigned m = __ballot_sync(kFull, key == c);
    if (key == c) slot = base + __popc(m & lt);
    base += __popc(m);
  };
  (one(Cs), ...);
  return base;
}

}  // namespace

// Parts of a batch one launch evaluates.  Large batches take two launches:
// PART_NEAR (in-grid and invalid points, alpha_s and the invalid count of
// every point; points that need a rule are skipped) and PART_FAR (only the
// points that need a rule: a range test on the bit patterns finds them, they
// wait in the per-class queues and run class-pure tiles).  Each kernel keeps
// a small loop: in one kernel the continuation code evicted the in-grid loop
// from the instruction cache (19% of stalls) and raised its register need.
enum { PART_ALL = 0, PART_NEAR = 1, PART_FAR = 2 };

// Class of a point that needs a continuation rule (C_LOWX..C_LOWX_LOWQ), or
// -1: the range tests of sites() on the raw bit patterns, nothing else.
__device__ __forceinline__ int far_class(const GridView &g, double x, double q2) {
  const long long kx = __double_as_longlong(x), kq = __double_as_longlong(q2);
  if (!(kq > 0 && kq < 0x7FF0000000000000LL && kx > 0 && kx <= __double_as_longlong(g.xlast))) return -1;
  const bool lowx = kx < __double_as_longlong(g.x0);
  const bool lowq = kq < __double_as_longlong(g.q2min), highq = kq > __double_as_longlong(g.q2max);
  if (!(lowx || lowq || highq)) return -1;
  return lowx ? (highq ? C_LOWX_HIGHQ : lowq ? C_LOWX_LOWQ : C_LOWX) : (highq ? C_HIGHQ : C_LOWQ);
}

// MODE_POINTS:  points xa[n], qa[n]; out[n][ncol] for columns col0..col0+ncol-1;
//               as_out[n] (alpha_s) when not null.
// MODE_MC:      events xa[n] (x1), xb[n] (x2), Q^2 = x1 x2 s; out[n][2 nf + 1]
//               (the flavours at x1, at x2, alpha_s); with gen.on the events
//               are generated (mc.cuh) and xa, xb are not read.
// MODE_MEMBERS: points xa[n], qa[n]; out[nmem][n][nf].  A warp's unit is
//               (tile, chunk of mchunk members); phase 1 repeats per chunk.
// One launch for everything (small batches) holds both the float-float
// positions and the continuation code: two blocks per SM give it the
// registers to do so without spilling.
template <int MODE, int PART>
__global__ void __launch_bounds__(kThreads, (PART == PART_ALL && MODE != MODE_MEMBERS) || PART == PART_FAR ? 2 : 3)
k_xf64(GridView g, const double *__restrict__ xa, const double *__restrict__ qa, const double *__restrict__ xb,
       double s, long long n, int col0, int ncol, int mchunk, double *__restrict__ out,
       double *__restrict__ as_out, McGen gen) {
  constexpr bool kQueue = MODE != MODE_MEMBERS && PART != PART_NEAR;
  extern __shared__ __align__(16) unsigned char smem[];
  size_t off = 0;
  long long *xkeys = reinterpret_cast<long long *>(smem + off);
  off += keys_bytes(g.nx, 8);
  long long *qkeys = reinterpret_cast<long long *>(smem + off);
  off += keys_bytes(g.nrows, 8);
  long long *akeys = reinterpret_cast<long long *>(smem + off);
  off += keys_bytes(g.na, 8);
  float4 *FTl = reinterpret_cast<float4 *>(smem + off);
  off += sizeof(float4) * kFFLogTab;
  float2 *FTe = reinterpret_cast<float2 *>(smem + off);
  off += sizeof(float2) * kFFExpTab;
  Rec64 *recs = reinterpret_cast<Rec64 *>(smem + off);
  off += kWarps * sizeof(Rec64);
  Queue64 *queues = reinterpret_cast<Queue64 *>(smem + off);

  const bool want_as = PART != PART_FAR && (MODE == MODE_MC || (MODE == MODE_POINTS && as_out != nullptr));
  load_keys<double>(g, xkeys, 0);
  load_keys<double>(g, qkeys, 1);
  if (want_as) load_keys<double>(g, akeys, 2);
  // positions and continuation sites in float-float (member sets keep the
  // FP64 logarithm: their grids have ffpos = 0, and the kernel is smaller
  // without the other path)
  const bool ffp = MODE != MODE_MEMBERS && g.ff && g.ffpos;
  // float-float positions (ffpos.cuh) of in-grid points, continued points'
  // sites and alpha_s: their steps table after the queues; then the FP64
  // logarithm's tables, which only a grid without float-float positions
  // reads (none reserved otherwise: xf64_smem)
  float4 *LF = reinterpret_cast<float4 *>(smem + off + (kQueue ? kWarps * sizeof(Queue64) : 0));
  float2 *LF2 = reinterpret_cast<float2 *>(LF + kLogTab);
  if (g.ffpos)
    for (int i = threadIdx.x; i < kLogTab; i += kThreads) { LF[i] = g.lnfff[i]; LF2[i] = g.lnfff2[i]; }
  // the per-knot position tables and cell maps (PosTabs) on grids with
  // float-float positions (member sets read them from global memory)
  const bool stp = MODE != MODE_MEMBERS && g.ffpos;
  unsigned char *tab = reinterpret_cast<unsigned char *>(LF2) + keys_bytes(kLogTab, 8);
  PosTabs PT = pos_tabs(g);
  if (stp) {
    float4 *xp = reinterpret_cast<float4 *>(tab), *qp = xp + g.nx, *ap = qp + g.nrows;
    double *ac = reinterpret_cast<double *>(ap + g.na);
    int *rq = reinterpret_cast<int *>(ac + 6 * g.na);
    for (int i = threadIdx.x; i < g.nx; i += kThreads) xp[i] = g.xposff[i];
    for (int i = threadIdx.x; i < g.nrows; i += kThreads) { qp[i] = g.qposff[i]; rq[i] = g.row_qc[i]; }
    if (want_as) {
      for (int i = threadIdx.x; i < g.na; i += kThreads) ap[i] = g.aposff[i];
      for (int i = threadIdx.x; i < 6 * g.na; i += kThreads) ac[i] = g.acell[i];
    }
    PT = PosTabs{xp, qp, ap, ac, rq};
    tab += pos_tabs_bytes(g.nx, g.nrows, g.na);
  }
  double2 *LTt = reinterpret_cast<double2 *>(tab);
  double *LTh = reinterpret_cast<double *>(LTt + kLogTab);
  if (!ffp)
    for (int i = threadIdx.x; i < kLogTab; i += kThreads) { LTt[i] = g.tlogtab[i]; LTh[i] = g.tloghtab[i]; }
  const LogTabs LT{LTt, LTh};
  for (int i = threadIdx.x; i < kFFLogTab; i += kThreads) FTl[i] = g.fflog[i];
  for (int i = threadIdx.x; i < kFFExpTab; i += kThreads) FTe[i] = g.ffexp[i];
  const FFTabs FT{FTl, FTe};
  const double *ET = g.texptab;  // the FP64 exponential (grids outside float-float range) reads it from L2
  __syncthreads();

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  Rec64 &R = recs[warp];
  Queue64 &Q = queues[warp];  // not touched for member sets (no room reserved)
  const int per_tile = MODE == MODE_MC ? 16 : 32;
  const int nc = MODE == MODE_MC ? g.nf : ncol;  // columns per point
  const int cbase = MODE == MODE_MC ? 0 : col0;
  const long long ntiles = (n + per_tile - 1) / per_tile;
  const int nchunks = MODE == MODE_MEMBERS ? (g.nmem + mchunk - 1) / mchunk : 1;
  const long long nunits = ntiles * nchunks;
  const long long nwarps = (long long)gridDim.x * kWarps;
  int nq[kFar] = {};  // queued continuation points per class (warp-uniform)

  // the point behind a queue entry: coordinates and output offset
  auto point_of = [&](unsigned id, double &x, double &q2, long long &ob) {
    if (MODE != MODE_MC) {
      x = xa[id];
      q2 = qa[id];
      ob = (long long)id * nc;
    } else {
      const unsigned long long e = id >> 1;
      double x1, x2;
      if (gen.on) mc_event(gen, e, x1, x2);
      else { x1 = xa[e]; x2 = xb[e]; }
      q2 = x1 * x2 * s;
      x = (id & 1) ? x2 : x1;
      ob = (long long)e * (2 * g.nf + 1) + (long long)(id & 1) * g.nf;
    }
  };
  // a tile of queued points of class C_LOWX + c: lane i takes entry from + i
  auto drain = [&](int c, int from, int cnt) {
    const bool present = lane < cnt;
    double x = 0.0, q2 = 0.0, lq;
    long long ob = 0;
    if (present) {
      point_of(Q.idx[c][from + lane], x, q2, ob);
    }
    int slot = 0, np;
    if (ffp) {  // warp-uniform: sites and rule parameters without the FP64 logarithm
      FarFF fs;
      fs.cls = -1;
      if (present) fs = far_sites_ff(g, xkeys, qkeys, LF, LF2, x, q2, PT);
      np = sort_slots<C_LOWX, C_HIGHQ, C_LOWQ, C_LOWX_HIGHQ, C_LOWX_LOWQ>(fs.cls, lane, slot);
      if (present) store_point_far_ff(R, slot, fs, ob, g);
    } else {
      PointSites<double> ps;
      ps.cls = -1;
      if (present) ps = sites(g, xkeys, qkeys, x, q2, LT, lq);
      np = sort_slots<C_LOWX, C_HIGHQ, C_LOWQ, C_LOWX_HIGHQ, C_LOWX_LOWQ>(ps.cls, lane, slot);
      if (present) store_point(R, slot, ps, ob, g.ff);
    }
    __syncwarp();
    items64<MODE == MODE_MC>(g, R, np, nc, cbase, 0, 0, out, LT, ET, FT, lane);
    __syncwarp();
  };

  // full tiles of one class; with last, also the partial ones (one call site
  // of the drain code)
  auto drain_ready = [&](bool last) {
    while (true) {
      int c0 = -1, from = 0, cnt = 0;
#pragma unroll
      for (int c = 0; c < kFar; c++)
        if (c0 < 0 && (nq[c] >= 32 || (last && nq[c] > 0))) {
          c0 = c;
          cnt = nq[c] < 32 ? nq[c] : 32;
          nq[c] -= cnt;
          from = nq[c];
        }
      if (c0 < 0) break;
      drain(c0, from, cnt);
    }
  };

  // one call site of the queue drain (it is inlined once): the loop runs one
  // more, empty round to drain the queues at the end
  for (long long unit = (long long)blockIdx.x * kWarps + warp;; unit += nwarps) {
    const bool more = unit < nunits;  // warp-uniform
    if (more) {
      const long long tile = unit / nchunks;
      const int chunk = (int)(unit - tile * nchunks);
      const long long e0 = tile * per_tile;
      const int ne = (int)(n - e0 < per_tile ? n - e0 : per_tile);

      // ---- phase 1: lane = point ----
      bool present;
      double x = 0.0, q2 = 0.0, lq = 0.0;
      long long ob;
      if (MODE != MODE_MC) {
        present = lane < ne;
        if (present) { x = xa[e0 + lane]; q2 = qa[e0 + lane]; }
        ob = (e0 + lane) * (long long)nc;
      } else {
        const int e = lane >> 1;
        present = e < ne;
        if (present) {
          double x1, x2;
          if (gen.on) mc_event(gen, (unsigned long long)(e0 + e), x1, x2);
          else { x1 = xa[e0 + e]; x2 = xb[e0 + e]; }
          q2 = x1 * x2 * s;
          x = (lane & 1) ? x2 : x1;
          if (PART != PART_FAR && gen.shat_out && (lane & 1) == 0) gen.shat_out[e0 + e] = q2;
          if (gen.cut && !(q2 >= gen.shat_min)) present = false;  // zero weight: not evaluated
        }
        ob = (e0 + e) * (long long)(2 * g.nf + 1) + (lane & 1) * g.nf;
      }
      if constexpr (PART == PART_FAR) {  // queue the points that need a rule, nothing else
        const int fc = present ? far_class(g, x, q2) : -1;
        const unsigned id = MODE == MODE_MC ? (unsigned)(2 * (e0 + (lane >> 1)) + (lane & 1)) : (unsigned)(e0 + lane);
#pragma unroll
        for (int c = 0; c < kFar; c++) {
          const unsigned fm = __ballot_sync(kFull, fc == C_LOWX + c);
          if (fc == C_LOWX + c) Q.idx[c][nq[c] + __popc(fm & ((1u << lane) - 1u))] = id;
          nq[c] += __popc(fm);
        }
        __syncwarp();
      }
      if constexpr (PART != PART_FAR) {
        PointSites<double> ps;
        ps.cls = -1;
        NearFF nf;
        nf.cls = -1;
        if (ffp) {  // warp-uniform
          // classification and in-grid positions without the FP64 logarithm;
          // continuation points keep the FP64 sites of their rules (the near
          // launch leaves them to the far one)
          if (present) nf = near_sites_ff(g, xkeys, qkeys, LF, LF2, x, q2, PT);
          ps.cls = nf.cls;
          if (PART != PART_NEAR && !kQueue && is_far(nf.cls)) ps = sites(g, xkeys, qkeys, x, q2, LT, lq);
        } else {
          if (present) ps = sites(g, xkeys, qkeys, x, q2, LT, lq);
          // in-grid points contract in float-float, except exact knot hits
          // (t = u = 0), which keep FP64 so that knot values come back bit-exact
          if (ps.cls == C_IN && g.ff &&
              !((__double_as_longlong(ps.t0) << 1) == 0 && (__double_as_longlong(ps.u0) << 1) == 0))
            ps.cls = C_INF;
        }
        if (MODE != MODE_MEMBERS || chunk == 0) {
          const unsigned inv = __ballot_sync(kFull, ps.cls == C_INVALID);
          if (lane == 0 && inv) atomicAdd(g.invalid, (unsigned long long)__popc(inv));
        }
        if (MODE == MODE_MC) {
          if (present && (lane & 1) == 0)
            out[ob + 2 * g.nf] = g.ffpos ? alphas_ff(g, akeys, LF, LF2, q2, PT) : alphas_eval(g, akeys, q2, lq);
        } else if (MODE == MODE_POINTS) {
          if (present && as_out) as_out[e0 + lane] = g.ffpos ? alphas_ff(g, akeys, LF, LF2, q2, PT) : alphas_eval(g, akeys, q2, lq);
        }

        int key = ps.cls, slot = 0, np;
        if (PART == PART_NEAR) {  // points that need a rule are the far launch's
          if (is_far(ps.cls)) key = -1;
          np = sort_slots<C_INF, C_IN, C_INVALID>(key, lane, slot);
        } else if (kQueue) {
          const unsigned id = MODE == MODE_MC ? (unsigned)(2 * (e0 + (lane >> 1)) + (lane & 1)) : (unsigned)(e0 + lane);
#pragma unroll
          for (int c = 0; c < kFar; c++) {
            const unsigned fm = __ballot_sync(kFull, ps.cls == C_LOWX + c);
            if (ps.cls == C_LOWX + c) {
              Q.idx[c][nq[c] + __popc(fm & ((1u << lane) - 1u))] = id;
              key = -1;
            }
            nq[c] += __popc(fm);
          }
          np = sort_slots<C_INF, C_IN, C_INVALID>(key, lane, slot);
        } else {
          np = sort_slots<C_INF, C_IN, C_LOWX, C_HIGHQ, C_LOWQ, C_LOWX_HIGHQ, C_LOWX_LOWQ, C_INVALID>(key, lane, slot);
        }
        if (key >= 0) {
          if (ffp && !is_far(ps.cls)) store_point_ff(R, slot, nf, ob);
          else store_point(R, slot, ps, ob, g.ff);
        }
        __syncwarp();

        // ---- phase 2: items ----
        if (MODE == MODE_MEMBERS) {
          const int m1 = min(g.nmem, (chunk + 1) * mchunk);
          for (int m = chunk * mchunk; m < m1; m++)
            items64<MODE == MODE_MC>(g, R, np, nc, cbase, m, (long long)m * n * nc, out, LT, ET, FT, lane);
        } else {
          items64<MODE == MODE_MC, PART != PART_NEAR>(g, R, np, nc, cbase, 0, 0, out, LT, ET, FT, lane);
        }
        __syncwarp();
      }
    }
    if (kQueue) drain_ready(!more);
    if (!more) break;
  }
}

static int num_sms() {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
  }
  return sms;
}

template <int MODE, int PART = PART_ALL>
static size_t xf64_smem(const GridView &g) {
  // as in the kernel: no FP64 log tables with float-float positions and
  // contraction; the position tables staged with float-float positions
  const bool ffp = MODE != MODE_MEMBERS && g.ff && g.ffpos, stp = MODE != MODE_MEMBERS && g.ffpos;
  return keys_bytes(g.nx, 8) + keys_bytes(g.nrows, 8) + keys_bytes(g.na, 8) + sizeof(float4) * kFFLogTab +
         sizeof(float2) * kFFExpTab +
         kWarps * (sizeof(Rec64) + (MODE == MODE_MEMBERS || PART == PART_NEAR ? 0 : sizeof(Queue64))) +
         sizeof(float4) * kLogTab + keys_bytes(kLogTab, 8) + (stp ? pos_tabs_bytes(g.nx, g.nrows, g.na) : 0) +
         (ffp ? 0 : sizeof(double2) * kLogTab + keys_bytes(kLogTab, 8));
}

// Batches of at least this many points take the two launches (near, far).
constexpr long long kSplitMin = 1LL << 16;

template <int MODE, int PART = PART_ALL>
static int launch_mode(const pdf_grid *grid, const double *xa, const double *qa, const double *xb, double s,
                       long long n, int col0, int ncol, double *out, double *as_out, const McGen &gen,
                       cudaStream_t st) {
  if constexpr (MODE != MODE_MEMBERS && PART == PART_ALL) {
    if (n >= kSplitMin) {
      const int rc = launch_mode<MODE, PART_NEAR>(grid, xa, qa, xb, s, n, col0, ncol, out, as_out, gen, st);
      if (rc) return rc;
      if (MODE == MODE_MC && gen.near_only) return PDF_OK;  // no event of the launch needs a rule
      return launch_mode<MODE, PART_FAR>(grid, xa, qa, xb, s, n, col0, ncol, out, as_out, gen, st);
    }
  }
  const GridView &g = grid->v;
  const size_t smem = xf64_smem<MODE, PART>(g);
  auto kern = k_xf64<MODE, PART>;
  static LaunchCache cache;
  const int per_sm = cache.blocks_per_sm(kern, kThreads, smem);
  const int per_tile = MODE == MODE_MC ? 16 : 32;
  const long long ntiles = (n + per_tile - 1) / per_tile;
  const long long cap = (long long)num_sms() * per_sm;
  // member sets: split the members into chunks until there are about two
  // units per resident warp (one chunk when the points alone suffice)
  int mchunk = 1;
  long long nunits = ntiles;
  if (MODE == MODE_MEMBERS) {
    const long long target = 2 * cap * kWarps;
    long long nchunks = (target + ntiles - 1) / ntiles;
    if (nchunks > g.nmem) nchunks = g.nmem;
    if (nchunks < 1) nchunks = 1;
    mchunk = (int)((g.nmem + nchunks - 1) / nchunks);
    nchunks = (g.nmem + mchunk - 1) / mchunk;
    nunits = ntiles * nchunks;
  }
  long long blocks = (nunits + kWarps - 1) / kWarps;
  if (blocks > cap) blocks = cap;
  kern<<<(unsigned)blocks, kThreads, smem, st>>>(g, xa, qa, xb, s, n, col0, ncol, mchunk, out, as_out, gen);
  return check_launch(MODE == MODE_MC ? "pdf_mc_event kernel" : "xfxq2 kernel (FP64)");
}

int launch_xf64(const pdf_grid *grid, int mode, const double *xa, const double *qa, const double *xb, double s,
                long long n, int col0, int ncol, double *out, double *as_out, cudaStream_t st, const McGen *gen) {
  McGen off{};
  const McGen &G = gen ? *gen : off;
  switch (mode) {
    case MODE_POINTS: return launch_mode<MODE_POINTS>(grid, xa, qa, xb, s, n, col0, ncol, out, as_out, off, st);
    case MODE_MC: return launch_mode<MODE_MC>(grid, xa, qa, xb, s, n, col0, ncol, out, nullptr, G, st);
    default: return launch_mode<MODE_MEMBERS>(grid, xa, qa, xb, s, n, col0, ncol, out, nullptr, off, st);
  }
}

}  // namespace pdfgb
