// sites.cuh -- per-point classification, cell search, patch-site positions
// and alpha_s, shared by the evaluation and adjoint kernels.
#pragma once

#include <cmath>

#include "pdf_internal.cuh"
#include "ffpos.cuh"

namespace pdfgb {

template <typename T>
struct Prec;
template <>
struct Prec<double> {
  using K = long long;
  static __device__ __forceinline__ K key(double v) { return __double_as_longlong(v); }
  static __device__ __forceinline__ const double *coef(const GridView &g) { return g.coef; }
};
template <>
struct Prec<float> {
  using K = int;
  static __device__ __forceinline__ K key(float v) { return __float_as_int(v); }
  static __device__ __forceinline__ const float *coef(const GridView &g) { return g.coef32; }
};

// Sites and continuation parameters of one point.  pq is the high-Q^2
// continuation parameter, or rho = Q^2/Q2min for the low-Q^2 classes.
// ts0 = 1 - t0 and us0 = 1 - u0, carried separately so that whichever of a
// position and its complement is small keeps its relative precision.
template <typename T>
struct PointSites {
  int cls, xc0, xc1, qc0, qc1;
  T t0, t1, u0, u1, ts0, us0, px, pq, lr;
};

// ---- FP64 classification and sites ---------------------------------------
// Range tests compare raw bit patterns: for positive doubles the integer
// order is the numeric order, and zero, negative values, infinities and NaN
// fail them exactly as the FP64 tests would, so the FP64 pipe is left to the
// logarithms and positions.  lq receives ln Q^2 whenever Q^2 is positive and
// finite (alpha_s needs it even where x is invalid).  LT: tlog's table.
__device__ __forceinline__ PointSites<double> sites(const GridView &g, const long long *xkeys,
                                                    const long long *qkeys, double x, double q2,
                                                    LogTabs LT, double &lq) {
  PointSites<double> r;
  r.xc0 = r.xc1 = r.qc0 = r.qc1 = 0;
  r.t0 = r.t1 = r.u0 = r.u1 = r.px = r.pq = r.lr = 0.0;
  r.ts0 = r.us0 = 1.0;
  const long long kx = __double_as_longlong(x), kq = __double_as_longlong(q2);
  const bool qv = kq > 0 && kq < 0x7FF0000000000000LL;
  lq = qv ? tlog(q2, LT) : 0.0;
  if (!(qv && kx > 0 && kx <= __double_as_longlong(g.xlast))) { r.cls = C_INVALID; return r; }
  const bool lowx = kx < __double_as_longlong(g.x0);
  const bool lowq = kq < __double_as_longlong(g.q2min), highq = kq > __double_as_longlong(g.q2max);
  const double lx = tlog(x, LT);
  if (!lowx) {
    int i = search_cell(xkeys, g.nx, g.xstep, kx);
    r.xc0 = i;
    const double2 c0 = *reinterpret_cast<const double2 *>(g.xcell + 4 * i);
    const double2 c1 = *reinterpret_cast<const double2 *>(g.xcell + 4 * i + 2);
    r.t0 = (lx - c0.x) * c0.y;
    r.ts0 = fma(c1.x - lx, c0.y, c1.y);
    // the larger one from the smaller (exact at both knots); t + ts ~ 1, so
    // at most one is negative and the integer order decides as FP64 would
    if (__double_as_longlong(r.t0) <= __double_as_longlong(r.ts0)) r.ts0 = 1.0 - r.t0;
    else r.t0 = 1.0 - r.ts0;
  } else {
    r.xc1 = 1;
    r.px = (lx - g.lx0) * g.idx0;
  }
  if (!lowq && !highq) {
    int j = search_cell(qkeys, g.nrows, g.qstep, kq);
    r.qc0 = g.row_qc[j];
    const double2 c0 = *reinterpret_cast<const double2 *>(g.qcell + 4 * j);
    const double2 c1 = *reinterpret_cast<const double2 *>(g.qcell + 4 * j + 2);
    r.u0 = (lq - c0.x) * c0.y;
    r.us0 = fma(c1.x - lq, c0.y, c1.y);
    if (__double_as_longlong(r.u0) <= __double_as_longlong(r.us0)) r.us0 = 1.0 - r.u0;
    else r.u0 = 1.0 - r.us0;
  } else if (highq) {
    r.qc0 = g.nqc;
    r.qc1 = g.top_qc;
    r.pq = -(lq - g.lq2max) * g.idq_top;
  } else {
    r.qc1 = g.q101_qc;
    r.u1 = g.q101_u;
    r.pq = q2 / g.q2min;
    r.lr = tlog(r.pq, LT);
  }
  r.cls = lowx ? (highq ? C_LOWX_HIGHQ : lowq ? C_LOWX_LOWQ : C_LOWX)
               : (highq ? C_HIGHQ : lowq ? C_LOWQ : C_IN);
  return r;
}

// The same for a grid with float-float positions (ffpos.cuh): an in-grid
// point's t, 1 - t, u, 1 - u from the bit patterns (no FP64 logarithm),
// rounded to doubles; any other point as sites() gives it.  lq is left 0 for
// in-grid points (their callers take alpha_s elsewhere).
__device__ __forceinline__ PointSites<double> sites_ffpos(const GridView &g, const long long *xkeys,
                                                          const long long *qkeys, const float4 *LF,
                                                          const float2 *LF2, double x, double q2, LogTabs LT,
                                                          double &lq) {
  const long long kx = __double_as_longlong(x), kq = __double_as_longlong(q2);
  const bool ingrid = kq >= __double_as_longlong(g.q2min) && kq <= __double_as_longlong(g.q2max) &&
                      kx >= __double_as_longlong(g.x0) && kx <= __double_as_longlong(g.xlast);
  if (!ingrid) return sites(g, xkeys, qkeys, x, q2, LT, lq);
  PointSites<double> r;
  lq = 0.0;
  r.cls = C_IN;
  r.xc1 = r.qc1 = 0;
  r.t1 = r.u1 = r.px = r.pq = r.lr = 0.0;
  const int i = search_cell(xkeys, g.nx, g.xstep, kx);
  const int j = search_cell(qkeys, g.nrows, g.qstep, kq);
  r.xc0 = i;
  r.qc0 = g.row_qc[j];
  ff2 t, ts, u, us;
  const bool xk1 = kx != xkeys[i], qk1 = kq != qkeys[j];
  ff_cell_pos2(kx, xkeys[i], xk1 ? xkeys[i + 1] : 0, g.xposff[i], xk1 ? g.xposff[i + 1] : make_float4(0.f, 0.f, 0.f, 0.f),
               LF, LF2, t, ts);
  ff_cell_pos2(kq, qkeys[j], qk1 ? qkeys[j + 1] : 0, g.qposff[j], qk1 ? g.qposff[j + 1] : make_float4(0.f, 0.f, 0.f, 0.f),
               LF, LF2, u, us);
  r.t0 = ff_to_d(t);
  r.ts0 = ff_to_d(ts);
  r.u0 = ff_to_d(u);
  r.us0 = ff_to_d(us);
  return r;
}

// ---- FP32 classification and sites -----------------------------------------
// The comparisons against rounded-up/down float thresholds decide exactly as
// FP64 comparisons of the float input against the FP64 knots would.  ln x
// enters only relative to the nearer end knot k of the cell,
//   ln(x / k) = log1p((x - kf) / kf) + ln(kf / k)   (kf = k rounded to float,
// x - kf exact for x within a factor 2 of kf), so the small one of t and
// 1 - t keeps its relative precision: where xf varies steeply (x -> 1, where
// (1 - x)^b makes the value sensitive to t) the position is still good to a
// float ulp.  No absolute logarithm of x is rounded to FP32.
// c: the cell's 8-float row of the FP32 cell table (shared memory in the
// evaluation kernel, which stages the table per block).
__device__ __forceinline__ void cell_pos32(const float *c, float v, float &t, float &ts) {
  const float4 a = *reinterpret_cast<const float4 *>(c);
  const float4 b = *(reinterpret_cast<const float4 *>(c) + 1);
  if (v < b.w) {
    t = (log1pf((v - a.x) * a.y) + a.z) * a.w;
    ts = 1.f - t;
  } else {
    // ln(v / k1) <= 0; far below k1 (a cell wider than a factor 4) the
    // complement 1 + z of z = (v - k1)/k1 is no longer precise, and the
    // quotient itself is taken instead
    const float z = (v - b.x) * b.y;
    ts = -((z > -0.5f ? log1pf(z) : logf(v * b.y)) + b.z) * a.w;
    t = 1.f - ts;
  }
}

// xcell, qcell, rowqc: the grid's xcell32, qcell32 and row_qc tables (or
// copies of them in shared memory).
__device__ __forceinline__ PointSites<float> sites(const GridView &g, const int *xkeys, const int *qkeys,
                                                   const float *xcell, const float *qcell, const int *rowqc,
                                                   float x, float q2) {
  PointSites<float> r;
  r.xc0 = r.xc1 = r.qc0 = r.qc1 = 0;
  r.t0 = r.t1 = r.u0 = r.u1 = r.px = r.pq = r.lr = 0.f;
  r.ts0 = r.us0 = 1.f;
  bool valid = (x > 0.f) && (x <= g.xlast_rd) && (q2 > 0.f) && (q2 < INFINITY);
  if (!valid) { r.cls = C_INVALID; return r; }
  bool lowx = x < g.x0_ru, lowq = q2 < g.q2min_ru, highq = q2 > g.q2max_rd;
  if (!lowx) {
    int i = search_cell(xkeys, g.nx, g.xstep, __float_as_int(x));
    r.xc0 = i;
    cell_pos32(xcell + 8 * i, x, r.t0, r.ts0);
  } else {
    r.xc1 = 1;
    r.px = logf(x * g.x0inv32) * g.idx0_32;
  }
  if (!lowq && !highq) {
    int j = search_cell(qkeys, g.nrows, g.qstep, __float_as_int(q2));
    r.qc0 = rowqc[j];
    cell_pos32(qcell + 8 * j, q2, r.u0, r.us0);
  } else if (highq) {
    r.qc0 = g.nqc;
    r.qc1 = g.top_qc;
    r.pq = -logf(q2 * g.q2maxinv32) * g.idq_top32;
  } else {
    r.qc1 = g.q101_qc;
    r.u1 = g.q101_u32;
    r.pq = q2 / g.q2min32;
    r.lr = logf(r.pq);
  }
  r.cls = lowx ? (highq ? C_LOWX_HIGHQ : lowq ? C_LOWX_LOWQ : C_LOWX)
               : (highq ? C_HIGHQ : lowq ? C_LOWQ : C_IN);
  return r;
}

// ---- alpha_s (Sec. 2.3): constant outside, log-cubic inside ----------------
// lq = ln Q^2 from tlog, used only inside the node range.
__device__ __forceinline__ double alphas_eval(const GridView &g, const long long *akeys, double q2, double lq) {
  const long long kq = __double_as_longlong(q2);
  if (!(kq > 0 && kq < 0x7FF0000000000000LL)) return NAN;
  if (kq < __double_as_longlong(g.aq2lo)) return g.as_lo;
  if (kq > __double_as_longlong(g.aq2hi)) return g.as_hi;
  int j = search_cell(akeys, g.na, g.astep, kq);
  const double *c = g.acell + 6 * j;
  double u = (lq - c[0]) * c[1];
  return fma(fma(fma(c[5], u, c[4]), u, c[3]), u, c[2]);
}
// acell: the grid's acell32 table (or a copy in shared memory).
__device__ __forceinline__ float alphas_eval(const GridView &g, const int *akeys, const float *acell, float q2) {
  if (!((q2 > 0.f) && (q2 < INFINITY))) return NAN;
  if (q2 < g.aq2lo_ru) return g.as_lo32;
  if (q2 > g.aq2hi_rd) return g.as_hi32;
  int j = search_cell(akeys, g.na, g.astep, __float_as_int(q2));
  const float *c = acell + 6 * j;
  float u = log1pf(fmaf(q2, c[0], -1.f)) * c[1];
  return fmaf(fmaf(fmaf(c[5], u, c[4]), u, c[3]), u, c[2]);
}

// The per-knot tables a point's float-float positions read -- {ln m, 1/d}
// pairs of the x knots, Q rows and alpha_s nodes, the row -> Q cell map and
// the alpha_s cells -- from global memory, or from copies in shared memory
// (the FP64 evaluation kernels: a warp's scattered reads of a few-KB table
// then take a few shared-memory wavefronts instead of one L1 wavefront per
// cache line touched).
struct PosTabs {
  const float4 *xpos, *qpos, *apos;
  const double *acell;
  const int *row_qc;
};
__device__ __forceinline__ PosTabs pos_tabs(const GridView &g) {
  return {g.xposff, g.qposff, g.aposff, g.acell, g.row_qc};
}
// Bytes of the shared-memory copies, in the order xpos, qpos, apos (float4),
// acell (6 doubles per node), row_qc (ints, rounded up to 16 bytes).
__host__ __device__ inline size_t pos_tabs_bytes(int nx, int nrows, int na) {
  return 16 * (size_t)(nx + nrows + na) + 48 * (size_t)na + (((size_t)nrows * 4 + 15) / 16) * 16;
}

// alpha_s (Sec. 2.3) with the node position from ffpos.cuh: constant
// outside, the cubic in FP64 from the position.
__device__ __forceinline__ double alphas_ff(const GridView &g, const long long *akeys, const float4 *LF,
                                            const float2 *LF2, double q2, const PosTabs &T) {
  const long long kq = __double_as_longlong(q2);
  if (!(kq > 0 && kq < 0x7FF0000000000000LL)) return NAN;
  if (kq < __double_as_longlong(g.aq2lo)) return g.as_lo;
  if (kq > __double_as_longlong(g.aq2hi)) return g.as_hi;
  const int k = search_cell(akeys, g.na, g.astep, kq);
  const double u = ff_to_d(ff_cell_pos(kq, akeys[k], T.apos[k], LF, LF2));
  const double *c = T.acell + 6 * k;
  return fma(fma(fma(c[5], u, c[4]), u, c[3]), u, c[2]);
}
template <typename T>
__device__ __forceinline__ void load_keys(const GridView &g, typename Prec<T>::K *keys, int which);

template <>
__device__ __forceinline__ void load_keys<double>(const GridView &g, long long *keys, int which) {
  const double *src = which == 0 ? g.xk : which == 1 ? g.q2k : g.aq2;
  int n = which == 0 ? g.nx : which == 1 ? g.nrows : g.na;
  for (int i = threadIdx.x; i < n; i += blockDim.x) keys[i] = __double_as_longlong(src[i]);
}
template <>
__device__ __forceinline__ void load_keys<float>(const GridView &g, int *keys, int which) {
  const float *src = which == 0 ? g.xthr32 : which == 1 ? g.q2thr32 : g.aq2thr32;
  int n = which == 0 ? g.nx : which == 1 ? g.nrows : g.na;
  for (int i = threadIdx.x; i < n; i += blockDim.x) keys[i] = __float_as_int(src[i]);
}

__host__ __device__ inline size_t keys_bytes(int nkeys, size_t ksize) {
  return ((nkeys * ksize + 15) / 16) * 16;
}


}  // namespace pdfgb
