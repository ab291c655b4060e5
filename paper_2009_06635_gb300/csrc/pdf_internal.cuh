// pdf_internal.cuh -- device-side layout of a staged grid and the helpers
// shared by the evaluation kernels.
//
// Layout in HBM (all staged once by pdf_load_grid, PDFFlow Sec. 2.2):
//   coef   [nqc+1][nx][nflav][16]  bicubic patch of every cell and flavour as
//          its 4x4 Bezier control points b[l*4 + k] (Bernstein basis in t,
//          the position inside the cell in ln x, index k; in u, ln Q^2,
//          index l).  One evaluation reads one contiguous, 128-byte aligned
//          block (FP64) or 64 bytes (FP32), instead of gathering 16 knots;
//          the Bernstein weights are non-negative and sum to one, so the
//          evaluation has no cancellation beyond that of the data.
//   coef32 the same control points rounded to FP32, [nqc+1][nx][4][nfp][4]
//          (row l = 0..3 of every flavour, then the next row; nfp = nflav
//          rounded up to 8, so every row block is whole 128-byte lines), so
//          one load instruction over the flavours of a point reads
//          consecutive rows of as few lines as possible.
//   coefff the same control points as float-float pairs (hi, lo), laid out
//          [nqc+1][nx][8][nfp][4]: control points m, m+1 (m even) of a
//          flavour as {hi_m, hi_m+1, lo_m, lo_m+1} (flavour stride nfp as for
//          coef32): one 16-byte load per pair, one load instruction over the
//          flavours of a point reads consecutive bytes of whole lines, and
//          the two high (low) parts share a register pair for packed f32x2
//          arithmetic.
//   xk/q2k raw knots, searched as integer bit patterns (positive doubles
//          order like their bits), so a cell choice never depends on a log.
//   xcell  per x cell {ln x_i, 1/d, ln x_{i+1}, 0}, d = ln x_{i+1} - ln x_i;
//          qcell likewise per cell-start row; row_qc maps a cell-start row
//          to its Q-cell index.  The position in a cell is carried as the
//          pair t = (ln x - ln x_i)/d, 1 - t = (ln x_{i+1} - ln x)/d, each
//          from its own knot, so the smaller keeps its relative precision.
//          One extra, degenerate cell sits on the last x knot and one on the
//          top Q knot ({ln knot, 0}: t = 0 there, and its patch holds only
//          that knot's column or row), so a query exactly on the last knot
//          returns the tabulated value exactly, like every other knot.
//   xW/qW  per cell, the 4 knot weights of the tangent-augmented Hermite
//          segment as cubics in t (u): w_a(t) = sum_k W[a][k] t^k.  The patch
//          of a cell is sum_ab w_a(t) w_b(u) f_ab; coef is that sum expanded.
#pragma once

#include <mutex>
#include <cstdint>
#include <cuda_runtime.h>

#include "pdf_gb300.h"
#include "tang.cuh"

namespace pdfgb {

// Class of a query point (decides which sites are evaluated and how the
// continuation combines them).
enum : int {
  C_IN = 0,          // inside the grid
  C_LOWX = 1,        // x < x0, Q^2 inside
  C_HIGHQ = 2,       // x inside, Q^2 > Q2max
  C_LOWQ = 3,        // x inside, Q^2 < Q2min
  C_LOWX_HIGHQ = 4,  // both
  C_LOWX_LOWQ = 5,
  C_INVALID = 6,
  C_INF = 7,         // inside, contraction in float-float (FP64 path, FP64-level accuracy)
  NCLASS = 8
};

// A place where the in-grid interpolant is evaluated: patch cell + position.
template <typename T>
struct Site {
  int xc, qc;
  T t, u;
};

struct GridView {
  int nx, nrows, nf, nxc, nqc, na, nsub;  // nxc, nqc: proper cells; slots are nx, nqc + 1
  int xstep, qstep, astep;  // largest power of two <= n-1 (binary search start)

  const double *xk, *q2k;     // raw knots (bit patterns searched)
  const double *xcell;        // [nx][4]
  const double *qcell;        // [nrows][4] (cell-start rows and the top row)
  const int *row_qc;          // [nrows]
  const int *qc_row;          // [nqc + 1] first row of each Q cell
  double *vals;               // [nrows][nx][nf] device copy of the knot values
  const double *coef;         // [nqc + 1][nx][nf][16]
  const float *coef32;        // [nqc + 1][nx][4][nfp][4]: row l of every flavour, then the next row
  const float2 *coefff;       // [nqc + 1][nx][8][nfp][4] float-float copy of coef (see above)
  int ff;                     // 1 if every control point is safe for float-float
  int nmem;                   // members (replicas) sharing the knots; member m's
  size_t mstride;             // control points start m * mstride elements further
  int nfp;                    // flavour stride of coef32 / coefff (nf rounded up to 8)
  size_t mstride_ff;          // member stride of coefff (float2 elements)
  const double *xW, *qW;      // [nx][16], [nqc + 1][16]
  const float *xthr32, *q2thr32;   // smallest float >= knot
  const float *xcell32, *qcell32;  // [n][8], see cell32 in grid.cu
  const double2 *tlogtab;     // [kLogTab] {1/F_j, ln F_j} (tang.cuh)
  const double *tloghtab;     // [kLogTab] ln(F_j / 2)
  const double *texptab;      // [kExpTab] 2^(k/256)

  // alpha_s
  const double *aq2;          // [na]
  const double *acell;        // [na][6] {lq_j, 1/dlq, a0, a1, a2, a3}
  const float *acell32;       // [na][6] {1/Q^2_j, 1/dlq, a0, a1, a2, a3}
  const float *aq2thr32;
  double as_lo, as_hi, aq2lo, aq2hi;
  float as_lo32, as_hi32;

  // classification (FP64) and float thresholds (FP32)
  double x0, xlast, q2min, q2max;
  float x0_ru, xlast_rd, q2min_ru, q2max_rd, aq2lo_ru, aq2hi_rd;
  // continuation parameters
  double lx0, idx0;           // p_x = (ln x - lx0) * idx0
  double lq2max, idq_top;     // p_q = -(ln Q^2 - lq2max) * idq_top
  double inv_q2min, ln101;    // ln 1.01
  float x0inv32, idx0_32, q2maxinv32, idq_top32, q2min32, ln101_32;
  // fixed sites: the second x knot is (cell 1, t = 0), Q2max is the
  // degenerate top cell at u = 0, the knot below it (top_qc, u = 0), and
  // 1.01 Q2min is (q101_qc, q101_u)
  int q101_qc, top_qc;
  double q101_u;
  float q101_u32;

  unsigned long long *invalid;
  // 1 / ln 1.01 (the low-Q^2 rule multiplies by it); last, so that adding it
  // left the offsets of the fields above as they were
  double iln101;
  float iln101_32;
  // float-float continuation (ffmath.cuh): its tables, and 1 / ln 1.01 as a pair
  const float4 *fflog;  // [kFFLogTab]
  const float2 *ffexp;  // [kFFExpTab]
  float iln101_ffh, iln101_ffl;
  // Float-float positions of in-grid points (ffpos.cuh): per x knot, Q row
  // and alpha_s node {ln m hi, lo, 1/d hi, lo} (m the knot's binary
  // significand in [1, 2), d the ln-width of the cell it starts, 0 where it
  // starts none), and per step F_j = 1 + j/256 {1/F_j hi, lo, ln F_j hi, lo}.
  // ffpos = 1 when every knot is a normal double, no cell spans 2^100 or
  // more (the exponent difference stays exact in floats) and the set has one
  // member (see load_impl in grid.cu).
  const float4 *xposff, *qposff, *aposff, *lnfff;
  int ffpos;
  const float2 *lnfff2;  // ln(F_j / 2) as a float pair (the high-significand steps)
  float q101ff[4];        // the 1.01 Q2min site's position u and 1 - u as float pairs
};

// ---------------------------------------------------------------------------
// search: largest index j in [0, n-1] with key_j <= key, given key_0 <= key
// (fixed-step binary search, no data-dependent trip count).  Keys are the bit
// patterns of positive floating-point numbers (monotone in the value).  With
// a repeated knot (a threshold) the later copy wins, which puts a query on
// the threshold into the upper subgrid; j = n-1 only for a query exactly on
// the last knot (its degenerate cell).
// ---------------------------------------------------------------------------
template <typename K>
__device__ __forceinline__ int search_cell(const K *keys, int n, int step, K key) {
  int lo = 0;
  for (int s = step; s > 0; s >>= 1) {
    int c = lo + s;
    if (c < n && keys[c] <= key) lo = c;
  }
  return lo;
}

// ---------------------------------------------------------------------------
// cubic Bernstein basis B_k(t) = C(3,k) t^k (1-t)^(3-k); B(0) = (1,0,0,0)
// exactly, so a site on a knot picks the control point (= knot value) alone.
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void bernstein(T t, T s, T *B) {  // s = 1 - t
  T t2 = t * t, s2 = s * s;
  B[0] = s2 * s;
  B[1] = T(3) * t * s2;
  B[2] = T(3) * t2 * s;
  B[3] = t2 * t;
}

// ---------------------------------------------------------------------------
// continuation rules (the EXTRAPOLATE box of PDFFlow Fig. 1)
// ---------------------------------------------------------------------------
// From g0 at one knot (p = 0) and g1 at the next one inwards (p = 1):
// log-linear if both are positive, linear otherwise.
__device__ __forceinline__ double pair_rule(double g0, double g1, double p, LogTabs LT, const double *ET) {
  if (__double_as_longlong(g0) > 0 && __double_as_longlong(g1) > 0)  // both > 0 (NaN: log-linear, NaN)
    return g0 * texp(p * tlog(ddiv(g1, g0), LT), ET);
  return g0 + (g1 - g0) * p;
}
__device__ __forceinline__ float pair_rule(float g0, float g1, float p) {
  if (g0 > 0.f && g1 > 0.f) return g0 * expf(p * logf(g1 / g0));
  return fmaf(g1 - g0, p, g0);
}

// Low Q^2: f0 = F(Q2min), f1 = F(1.01 Q2min); rho = Q^2/Q2min, lr = ln rho.
__device__ __forceinline__ double lowq_rule(double f0, double f1, double rho, double lr,
                                            double ln101, LogTabs LT, const double *ET) {
  double gam =
      (__double_as_longlong(f0) > 0 && __double_as_longlong(f1) > 0) ? tlog(ddiv(f1, f0), LT) / ln101 : 1.0;
  double ex = (gam * rho + 1.0) - rho;
  return f0 * texp(ex * lr, ET);
}
// The same with 1 / ln 1.01 given (a multiplication instead of the division).
__device__ __forceinline__ double lowq_rule_r(double f0, double f1, double rho, double lr,
                                              double iln101, LogTabs LT, const double *ET) {
  double gam =
      (__double_as_longlong(f0) > 0 && __double_as_longlong(f1) > 0) ? tlog(ddiv(f1, f0), LT) * iln101 : 1.0;
  double ex = (gam * rho + 1.0) - rho;
  return f0 * texp(ex * lr, ET);
}
__device__ __forceinline__ float lowq_rule(float f0, float f1, float rho, float lr, float iln101) {
  float gam = (f0 > 0.f && f1 > 0.f) ? logf(f1 / f0) * iln101 : 1.f;
  float ex = (gam * rho + 1.f) - rho;
  return f0 * expf(ex * lr);
}

// Combine the site values of one point and flavour according to its class.
// F(a, b) is the patch at x-site a (0/1) and q-site b (0/1).
template <typename T, typename FN>
__device__ __forceinline__ T combine(int cls, T px, T pq, T lr, T iln101, FN F) {
  switch (cls) {
    case C_IN: return F(0, 0);
    case C_LOWX: return pair_rule(F(0, 0), F(1, 0), px);
    case C_HIGHQ: return pair_rule(F(0, 0), F(0, 1), pq);
    case C_LOWQ: return lowq_rule(F(0, 0), F(0, 1), pq, lr, iln101);
    case C_LOWX_HIGHQ:
      return pair_rule(pair_rule(F(0, 0), F(0, 1), pq), pair_rule(F(1, 0), F(1, 1), pq), px);
    case C_LOWX_LOWQ:
      return pair_rule(lowq_rule(F(0, 0), F(0, 1), pq, lr, iln101),
                       lowq_rule(F(1, 0), F(1, 1), pq, lr, iln101), px);
    default: return T(NAN);
  }
}

// Host-side helpers shared by the translation units.
int set_error(int code, const char *fmt, ...);
int check_launch(const char *what);

// Blocks per SM of a kernel at a dynamic shared-memory size, found once per
// size (a small launch would otherwise pay for the attribute and occupancy
// queries on every call).  The size attribute only grows, so concurrent
// callers never lower it under one another's launch.  One device per process.
// A failed attribute or occupancy query (e.g. more shared memory than the
// device allows) counts as 0 blocks: callers with another kernel to fall back
// on pass at_least_one = false and see the 0; the others get 1 and let the
// launch report the error.
struct LaunchCache {
  std::mutex mu;
  size_t attr = 0, sizes[16] = {};
  int occ[16] = {}, nc = 0;
  template <typename K>
  int blocks_per_sm(K kern, int threads, size_t smem, bool at_least_one = true) {
    std::lock_guard<std::mutex> lock(mu);
    for (int i = 0; i < nc; i++)
      if (sizes[i] == smem) return at_least_one && occ[i] < 1 ? 1 : occ[i];
    int per_sm = 0;
    bool ok = true;
    if (smem > attr) {
      ok = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) == cudaSuccess;
      if (ok) attr = smem;
    }
    if (ok) ok = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem) == cudaSuccess;
    if (!ok) {
      cudaGetLastError();
      per_sm = 0;
    }
    const int slot = nc < 16 ? nc++ : 15;
    sizes[slot] = smem;
    occ[slot] = per_sm;
    return at_least_one && per_sm < 1 ? 1 : per_sm;
  }
};

// Process-wide bound on the stream-ordered device scratch one call may take
// for a sorted path (pdf_set_scratch_limit; default: none).
size_t scratch_limit();
// The per-device memory pool the sorted paths take their scratch from (kept
// between calls up to 256 MB), or nullptr.
cudaMemPool_t sort_pool(int dev);

// Evaluation layouts (see the kernels in xf64.cu and xfxq2.cu).
enum { MODE_POINTS = 0, MODE_MC = 1, MODE_MEMBERS = 2 };

}  // namespace pdfgb

// The opaque handle.
struct pdf_grid {
  pdfgb::GridView v;
  int *ffbad;  // device flag: a control point is outside the float-float range
  int device;
  int pids[PDF_MAX_NFLAV];
  // device allocations owned by the handle
  void *blocks[32];
  int nblocks;
  // host-I/O pipeline (lazily created): kIoStreams streams, one staging buffer each;
  // io_mu serialises the calls that use it (and mc_mu those that use the MC scratch)
  std::mutex io_mu, mc_mu;
  static constexpr int kIoStreams = 3;
  cudaStream_t io_stream[kIoStreams];
  cudaEvent_t io_event[kIoStreams];
  void *io_buf[kIoStreams];
  size_t io_cap;  // points per buffer
  // Monte Carlo integration scratch (lazily created): event rows, per-block
  // partial sums, the running sums
  double *mc_buf;
  size_t mc_cap;  // events per chunk the buffer holds
  double *mc_part, *mc_acc;
};

namespace pdfgb {
// FP64 evaluation (xf64.cu), mode = MODE_*: points xa, qa (columns
// col0..col0+ncol-1; alpha_s into as_out when not null), events xa, xb with
// Q^2 = xa xb s, or every member of the set.  Arguments already validated.
// With gen (MODE_MC only) the events are generated on the device (mc.cuh).
struct McGen;
int launch_xf64(const pdf_grid *grid, int mode, const double *xa, const double *qa, const double *xb, double s,
                long long n, int col0, int ncol, double *out, double *as_out, cudaStream_t st,
                const McGen *gen = nullptr);
// xfxq2.cu: all flavours (+ alpha_s when as_out is not null) in one pass.
int launch_all_f64(const pdf_grid *g, const double *x, const double *q2, long long n, double *out,
                   double *as_out, cudaStream_t st);
}  // namespace pdfgb
