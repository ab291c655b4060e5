// xfxq2.cu -- evaluation kernels for x f(x, Q^2) and alpha_s(Q^2).
//
// One warp owns a tile of 32 query points (16 events in the Monte Carlo
// layout).  Phase 1 (lane = point): read x and Q^2 (coalesced), classify
// against the grid edges, search the cells on the raw bit patterns (knots in
// shared memory), take ln x and ln Q^2 once, and record the Bernstein weights
// of the patch sites and the continuation parameters of the point; points
// are then ordered by class so that lanes of one instruction take the same
// branch.  Phase 2 (items = (point, flavour)): contract the weights with the
// cell's 16 control points, combine the sites by class, write the output.
//   FP64: one lane per item, 16 FMAs on weight products formed once per
//         point (the FP64 pipe is the bottleneck on GB300, so per-item FP64
//         work is kept minimal; sites on knots collapse to 4- or 1-term sums).
//   FP32: four lanes per item, each loading one float4 row of control
//         points, reduced with two shuffles: one load instruction covers
//         eight items, 512 contiguous bytes (the FP32 path is bound by the
//         L1/L2 gather, not arithmetic).
// Consecutive items are consecutive outputs, so [n][nflav] stores coalesce.
#include <cmath>
#include <type_traits>

#include "sites.cuh"

namespace pdfgb {

constexpr int kWarps = 8;
constexpr int kThreads = 32 * kWarps;

// Per-warp record of the points of one tile, indexed by class-sorted slot.
// W holds, per slot: for FP64 in-grid points the 16 products Bx[k] Bq[l] at
// [l*4 + k]; otherwise (and always for FP32) Bx0 | Bx1 | Bq0 | Bq1.
template <typename T>
struct WarpRec {
  int cls[32], orig[32], xc0[32], xc1[32], qc0[32], qc1[32];
  int off4[32];  // FP32 in-grid points: float4 offset of the cell's first flavour block
  T W[16][33];  // padded: rows of one slot fall in different banks
  T px[32], pq[32], lr[32], as[32];
};

enum { MODE_POINTS = 0, MODE_MC = 1, MODE_MEMBERS = 2 };

// ---- float-float arithmetic (a value is hi + lo, two floats, ~48 bits) -----
// Error-free product (FMA) and sum (TwoSum); the _rn intrinsics keep the
// compiler from contracting or reordering the error terms.
struct ff2 {
  float h, l;
};
__device__ __forceinline__ ff2 ff_of(double a) {
  float h = __double2float_rn(a);
  return {h, __double2float_rn(a - (double)h)};
}
__device__ __forceinline__ ff2 ff_mul(ff2 a, ff2 b) {
  float p = __fmul_rn(a.h, b.h);
  float e = __fmaf_rn(a.h, b.h, -p);
  e = __fmaf_rn(a.h, b.l, __fmaf_rn(a.l, b.h, e));
  float h = __fadd_rn(p, e);
  return {h, __fsub_rn(e, __fsub_rn(h, p))};
}
__device__ __forceinline__ void ff_bernstein(double t, double s, ff2 *B) {
  const ff2 tf = ff_of(t), sf = ff_of(s), three = {3.f, 0.f};
  const ff2 t2 = ff_mul(tf, tf), s2 = ff_mul(sf, sf);
  B[0] = ff_mul(s2, sf);
  B[1] = ff_mul(three, ff_mul(tf, s2));
  B[2] = ff_mul(three, ff_mul(t2, sf));
  B[3] = ff_mul(t2, tf);
}
// sum_m w_m b_m with w (hi, lo) from the record and b (hi, lo) from the
// float-float control points: exact products, TwoSum accumulation, the
// cross terms and the rounding errors gathered in a second float.
__device__ __forceinline__ double dot_ff16(const float2 *c, const double (*W)[33], int p) {
  const float4 *q = reinterpret_cast<const float4 *>(c);
  float sh = 0.f, sl = 0.f;
#pragma unroll
  for (int m2 = 0; m2 < 8; m2++) {
    const float4 v = __ldg(q + m2);
#pragma unroll
    for (int half = 0; half < 2; half++) {
      const float bh = half ? v.z : v.x, bl = half ? v.w : v.y;
      const float2 w = *reinterpret_cast<const float2 *>(&W[2 * m2 + half][p]);
      const float ph = __fmul_rn(w.x, bh);
      float pe = __fmaf_rn(w.x, bh, -ph);
      pe = __fmaf_rn(w.x, bl, __fmaf_rn(w.y, bh, pe));
      const float t = __fadd_rn(sh, ph);
      const float bp = __fsub_rn(t, sh);
      const float err = __fadd_rn(__fsub_rn(sh, __fsub_rn(t, bp)), __fsub_rn(ph, bp));
      sh = t;
      sl = __fadd_rn(sl, __fadd_rn(err, pe));
    }
  }
  return (double)sh + (double)sl;
}

// ---- FP64 item evaluation (one lane per item) ----------------------------
__device__ __forceinline__ double dot_w16(const double *c, const WarpRec<double> &R, int p) {
  const double2 *q = reinterpret_cast<const double2 *>(c);
  double2 v = __ldg(q);
  double acc = R.W[0][p] * v.x;
  acc = fma(R.W[1][p], v.y, acc);
#pragma unroll
  for (int m = 1; m < 8; m++) {
    v = __ldg(q + m);
    acc = fma(R.W[2 * m][p], v.x, acc);
    acc = fma(R.W[2 * m + 1][p], v.y, acc);
  }
  return acc;
}
// site with t general, u general: sum_l Bq[l] sum_k Bx[k] b[l][k]
__device__ __forceinline__ double site_tu(const double *c, const WarpRec<double> &R, int p, int a, int b) {
  double f = 0.0;
#pragma unroll
  for (int l = 0; l < 4; l++) {
    const double2 *q = reinterpret_cast<const double2 *>(c + 4 * l);
    double2 v0 = __ldg(q), v1 = __ldg(q + 1);
    double r = R.W[4 * a][p] * v0.x;
    r = fma(R.W[4 * a + 1][p], v0.y, r);
    r = fma(R.W[4 * a + 2][p], v1.x, r);
    r = fma(R.W[4 * a + 3][p], v1.y, r);
    f = l == 0 ? R.W[8 + 4 * b][p] * r : fma(R.W[8 + 4 * b + l][p], r, f);
  }
  return f;
}
// site on an x knot (t = 0): sum_l Bq[l] b[l][0]
__device__ __forceinline__ double site_u(const double *c, const WarpRec<double> &R, int p, int b) {
  double f = R.W[8 + 4 * b][p] * __ldg(c);
  f = fma(R.W[8 + 4 * b + 1][p], __ldg(c + 4), f);
  f = fma(R.W[8 + 4 * b + 2][p], __ldg(c + 8), f);
  return fma(R.W[8 + 4 * b + 3][p], __ldg(c + 12), f);
}
// site on a Q knot (u = 0): sum_k Bx[k] b[0][k]
__device__ __forceinline__ double site_t(const double *c, const WarpRec<double> &R, int p, int a) {
  const double2 *q = reinterpret_cast<const double2 *>(c);
  double2 v0 = __ldg(q), v1 = __ldg(q + 1);
  double f = R.W[4 * a][p] * v0.x;
  f = fma(R.W[4 * a + 1][p], v0.y, f);
  f = fma(R.W[4 * a + 2][p], v1.x, f);
  return fma(R.W[4 * a + 3][p], v1.y, f);
}

__device__ __forceinline__ double eval_item64(const GridView &g, const WarpRec<double> &R, int p, int col,
                                              size_t moff = 0) {
  const double *cb = g.coef + moff + (size_t)col * 16;
  const size_t stride = (size_t)g.nf * 16;
  auto C = [&](int a, int b) {
    int xc = a ? R.xc1[p] : R.xc0[p];
    int qc = b ? R.qc1[p] : R.qc0[p];
    return cb + ((size_t)qc * g.nx + xc) * stride;
  };
  switch (R.cls[p]) {
    case C_INF: {
      const int xc = R.xc0[p], qc = R.qc0[p];
      return dot_ff16(g.coefff + moff + (((size_t)qc * g.nx + xc) * g.nf + col) * 16, R.W, p);
    }
    case C_IN: return dot_w16(C(0, 0), R, p);
    case C_LOWX:  // sites (x0, Q^2), (x1, Q^2): t = 0
      return pair_rule(site_u(C(0, 0), R, p, 0), site_u(C(1, 0), R, p, 0), R.px[p]);
    case C_HIGHQ:  // sites (x, Q2max), (x, knot below): u = 0
      return pair_rule(site_t(C(0, 0), R, p, 0), site_t(C(0, 1), R, p, 0), R.pq[p]);
    case C_LOWQ:  // sites (x, Q2min): u = 0; (x, 1.01 Q2min): general
      return lowq_rule(site_t(C(0, 0), R, p, 0), site_tu(C(0, 1), R, p, 0, 1), R.pq[p], R.lr[p], g.ln101);
    case C_LOWX_HIGHQ: {  // all four sites are knots
      double a = pair_rule(__ldg(C(0, 0)), __ldg(C(0, 1)), R.pq[p]);
      double b = pair_rule(__ldg(C(1, 0)), __ldg(C(1, 1)), R.pq[p]);
      return pair_rule(a, b, R.px[p]);
    }
    case C_LOWX_LOWQ: {
      double a = lowq_rule(__ldg(C(0, 0)), site_u(C(0, 1), R, p, 1), R.pq[p], R.lr[p], g.ln101);
      double b = lowq_rule(__ldg(C(1, 0)), site_u(C(1, 1), R, p, 1), R.pq[p], R.lr[p], g.ln101);
      return pair_rule(a, b, R.px[p]);
    }
    default: return NAN;
  }
}

// ---- FP32 evaluation -------------------------------------------------------
// One lane, whole patch: sum_l Bq[l] sum_k Bx[k] b[l][k] (four float4 rows),
// rounded in the same order as the four-lane version ((p0 + p1) + (p2 + p3)),
// so one flavour alone and all flavours give identical bits.
__device__ __forceinline__ float site32_full(const float *c, const WarpRec<float> &R, int p, int a, int b) {
  const float4 *q = reinterpret_cast<const float4 *>(c);
  float pl[4];
#pragma unroll
  for (int l = 0; l < 4; l++) {
    float4 v = __ldg(q + l);
    float rr = R.W[4 * a][p] * v.x;
    rr = fmaf(R.W[4 * a + 1][p], v.y, rr);
    rr = fmaf(R.W[4 * a + 2][p], v.z, rr);
    rr = fmaf(R.W[4 * a + 3][p], v.w, rr);
    pl[l] = __fmul_rn(rr, R.W[8 + 4 * b + l][p]);
  }
  return (pl[0] + pl[1]) + (pl[2] + pl[3]);
}

__device__ __forceinline__ float eval_point32(const GridView &g, const WarpRec<float> &R, int p, int col) {
  const float *cb = g.coef32 + (size_t)col * 16;
  const size_t stride = (size_t)g.nf * 16;
  auto F = [&](int a, int b) {
    int xc = a ? R.xc1[p] : R.xc0[p];
    int qc = b ? R.qc1[p] : R.qc0[p];
    return site32_full(cb + ((size_t)qc * g.nx + xc) * stride, R, p, a, b);
  };
  return combine<float>(R.cls[p], R.px[p], R.pq[p], R.lr[p], g.ln101_32, F);
}

// Four lanes per item, lane r owns row l = r of the control points.
__device__ __forceinline__ float site32(const float *c, const WarpRec<float> &R, int p, int a, int b,
                                        int r, unsigned gm) {
  float4 v = __ldg(reinterpret_cast<const float4 *>(c) + r);
  float part = R.W[4 * a][p] * v.x;
  part = fmaf(R.W[4 * a + 1][p], v.y, part);
  part = fmaf(R.W[4 * a + 2][p], v.z, part);
  part = fmaf(R.W[4 * a + 3][p], v.w, part);
  part = __fmul_rn(part, R.W[8 + 4 * b + r][p]);
  part += __shfl_xor_sync(gm, part, 1);
  part += __shfl_xor_sync(gm, part, 2);
  return part;
}

__device__ __forceinline__ float eval_item32(const GridView &g, const WarpRec<float> &R, int p, int col,
                                             int r, unsigned gm) {
  const float *cb = g.coef32 + (size_t)col * 16;
  const size_t stride = (size_t)g.nf * 16;
  auto F = [&](int a, int b) {
    int xc = a ? R.xc1[p] : R.xc0[p];
    int qc = b ? R.qc1[p] : R.qc0[p];
    return site32(cb + ((size_t)qc * g.nx + xc) * stride, R, p, a, b, r, gm);
  };
  return combine<float>(R.cls[p], R.px[p], R.pq[p], R.lr[p], g.ln101_32, F);
}

// Write the Bernstein weights of a point's sites into its record slot.
template <typename T>
__device__ __forceinline__ void store_weights(WarpRec<T> &R, int slot, const PointSites<T> &ps,
                                              const GridView &g) {
  if (sizeof(T) == 8 && ps.cls == C_INF) {  // float-float weights for the FP64 contraction
    ff2 bx[4], bq[4];
    ff_bernstein((double)ps.t0, (double)ps.ts0, bx);
    ff_bernstein((double)ps.u0, (double)ps.us0, bq);
#pragma unroll
    for (int l = 0; l < 4; l++)
#pragma unroll
      for (int k = 0; k < 4; k++) {
        const ff2 w = ff_mul(bx[k], bq[l]);
        float2 *slot_ptr = reinterpret_cast<float2 *>(&R.W[l * 4 + k][slot]);
        *slot_ptr = make_float2(w.h, w.l);
      }
    return;
  }
  T bx0[4], bx1[4], bq0[4], bq1[4];
  bernstein<T>(ps.t0, ps.ts0, bx0);
  bernstein<T>(ps.t1, T(1) - ps.t1, bx1);
  bernstein<T>(ps.u0, ps.us0, bq0);
  bernstein<T>(ps.u1, T(1) - ps.u1, bq1);
  if (sizeof(T) == 8 && ps.cls == C_IN) {
#pragma unroll
    for (int l = 0; l < 4; l++)
#pragma unroll
      for (int k = 0; k < 4; k++) R.W[l * 4 + k][slot] = bx0[k] * bq0[l];
  } else {
#pragma unroll
    for (int k = 0; k < 4; k++) {
      R.W[k][slot] = bx0[k];
      R.W[4 + k][slot] = bx1[k];
      R.W[8 + k][slot] = bq0[k];
      R.W[12 + k][slot] = bq1[k];
    }
  }
}

// MODE_POINTS:  points xa[n], qa[n]; out[n][ncol] for columns col0..col0+ncol-1.
// MODE_MC:      events xa[n] (x1), xb[n] (x2), Q^2 = x1 x2 s; out[n][2 nf + 1].
// MODE_MEMBERS: points xa[n], qa[n]; out[nmem][n][nf], FP64 only.  A warp's
//               unit is (tile, chunk of mchunk members), so a few points times
//               many members still fill the GPU; phase 1 repeats per chunk.
template <typename T, int MODE>
__global__ void __launch_bounds__(kThreads, sizeof(T) == 8 ? 3 : 4)
k_xf(GridView g, const T *__restrict__ xa, const T *__restrict__ qa, const T *__restrict__ xb,
     T s, long long n, int col0, int ncol, int mchunk, T *__restrict__ out) {
  using K = typename Prec<T>::K;
  constexpr int LPI = sizeof(T) == 8 ? 1 : 4;  // lanes per item
  constexpr int IPI = 32 / LPI;                // items per warp instruction (FP64 loop)
  extern __shared__ __align__(16) unsigned char smem[];
  K *xkeys = reinterpret_cast<K *>(smem);
  K *qkeys = reinterpret_cast<K *>(smem + keys_bytes(g.nx, sizeof(K)));
  K *akeys = reinterpret_cast<K *>(smem + keys_bytes(g.nx, sizeof(K)) + keys_bytes(g.nrows, sizeof(K)));
  size_t rec_off = keys_bytes(g.nx, sizeof(K)) + keys_bytes(g.nrows, sizeof(K)) +
                   (MODE == MODE_MC ? keys_bytes(g.na, sizeof(K)) : 0);
  WarpRec<T> *recs = reinterpret_cast<WarpRec<T> *>(smem + rec_off);
  load_keys<T>(g, xkeys, 0);
  load_keys<T>(g, qkeys, 1);
  if (MODE == MODE_MC) load_keys<T>(g, akeys, 2);
  __syncthreads();

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  WarpRec<T> &R = recs[warp];
  const int per_tile = MODE == MODE_MC ? 16 : 32;
  const int per = MODE == MODE_MC ? 2 * g.nf + 1 : ncol;  // outputs per tile unit
  const int dp = IPI / per, dc = IPI - dp * per;
  const int r = lane & (LPI - 1);
  const unsigned gm = LPI == 1 ? 1u << lane : 0xFu << (lane & ~3);
  const long long ntiles = (n + per_tile - 1) / per_tile;
  const int nchunks = MODE == MODE_MEMBERS ? (g.nmem + mchunk - 1) / mchunk : 1;
  const long long nunits = ntiles * nchunks;
  const long long nwarps = (long long)gridDim.x * kWarps;

  for (long long unit = (long long)blockIdx.x * kWarps + warp; unit < nunits; unit += nwarps) {
    const long long tile = unit / nchunks;
    const int chunk = (int)(unit - tile * nchunks);
    const long long e0 = tile * per_tile;
    const int ne = (int)(n - e0 < per_tile ? n - e0 : per_tile);

    // ---- phase 1: lane = point ----
    bool present;
    T x = T(0), q2 = T(0);
    if (MODE != MODE_MC) {  // points (also member sets): xa[n], qa[n]
      present = lane < ne;
      if (present) { x = xa[e0 + lane]; q2 = qa[e0 + lane]; }
    } else {  // events: x1 = xa, x2 = xb
      const int e = lane >> 1;
      present = e < ne;
      if (present) {
        T x1 = xa[e0 + e], x2 = xb[e0 + e];
        q2 = x1 * x2 * s;
        x = (lane & 1) ? x2 : x1;
      }
    }
    PointSites<T> ps;
    ps.cls = NCLASS;
    if (present) ps = sites(g, xkeys, qkeys, x, q2);
    // FP64 in-grid points contract in float-float, except exact knot hits
    // (t = u = 0), which keep the FP64 path so that knots stay bit-exact
    if (sizeof(T) == 8 && ps.cls == C_IN && g.ff && !(ps.t0 == T(0) && ps.u0 == T(0))) ps.cls = C_INF;
    unsigned inv = __ballot_sync(0xffffffffu, present && ps.cls == C_INVALID);
    if (lane == 0 && inv) atomicAdd(g.invalid, (unsigned long long)__popc(inv));

    int slot = lane;
    if (MODE != MODE_MC) {  // order points by class (counting sort over the warp)
      int base = 0;
      const unsigned lt = (1u << lane) - 1u;
#pragma unroll
      for (int c = 0; c <= NCLASS; c++) {
        unsigned m = __ballot_sync(0xffffffffu, ps.cls == c);
        if (ps.cls == c) slot = base + __popc(m & lt);
        base += __popc(m);
      }
    }
    R.cls[slot] = ps.cls; R.orig[slot] = lane;
    if (sizeof(T) == 4) R.off4[slot] = ((ps.qc0 * g.nx + ps.xc0) * g.nf + col0) * 4;
    R.xc0[slot] = ps.xc0; R.xc1[slot] = ps.xc1; R.qc0[slot] = ps.qc0; R.qc1[slot] = ps.qc1;
    R.px[slot] = ps.px; R.pq[slot] = ps.pq; R.lr[slot] = ps.lr;
    if (present && ps.cls != C_INVALID) store_weights<T>(R, slot, ps, g);
    if (MODE == MODE_MC && (lane & 1) == 0) R.as[lane >> 1] = present ? alphas_eval(g, akeys, q2) : T(0);
    __syncwarp();

    // ---- phase 2, FP32: per point, lanes over (column, row) ----
    if constexpr (sizeof(T) == 4) {
      const WarpRec<float> &RF = reinterpret_cast<const WarpRec<float> &>(R);
      if (MODE == MODE_POINTS && ncol == 1) {  // one column: a lane per point
        if (lane < ne) out[e0 + RF.orig[lane]] = eval_point32(g, RF, lane, col0);
      } else {
        const int nc = MODE == MODE_MC ? g.nf : ncol;
        const int npts = MODE == MODE_MC ? 2 * ne : ne;
        for (int q = 0; q < npts; q++) {  // warp-uniform: no divergence by class
          const long long ob = MODE == MODE_POINTS ? (e0 + RF.orig[q]) * (long long)ncol
                                                   : (e0 + (q >> 1)) * (long long)per + (q & 1) * g.nf;
          if (RF.cls[q] == C_IN) {
            // the point's column blocks are contiguous: lane k owns rows 2h, 2h+1
            // (h = k & 1) of column k >> 1, 32 bytes at cell_base + 8 k floats
            const float4 *cbp = reinterpret_cast<const float4 *>(g.coef32) + RF.off4[q];
            const float b0 = RF.W[0][q], b1 = RF.W[1][q], b2 = RF.W[2][q], b3 = RF.W[3][q];
            const int hr = lane & 1;
            const float bqa = RF.W[8 + 2 * hr][q], bqb = RF.W[9 + 2 * hr][q];
            const unsigned pm = 3u << (lane & 30);
            for (int k = lane; k < 2 * nc; k += 32) {
              const float4 v0 = __ldg(cbp + 2 * k), v1 = __ldg(cbp + 2 * k + 1);
              float ra = b0 * v0.x;
              ra = fmaf(b1, v0.y, ra);
              ra = fmaf(b2, v0.z, ra);
              ra = fmaf(b3, v0.w, ra);
              float rb = b0 * v1.x;
              rb = fmaf(b1, v1.y, rb);
              rb = fmaf(b2, v1.z, rb);
              rb = fmaf(b3, v1.w, rb);
              // (p0 + p1) + (p2 + p3), the order of every FP32 patch sum
              float part = __fadd_rn(__fmul_rn(ra, bqa), __fmul_rn(rb, bqb));
              const float other = __shfl_xor_sync(pm, part, 1);
              if (hr == 0) out[ob + (k >> 1)] = __fadd_rn(part, other);
            }
          } else {
            for (int k = lane; k < 4 * nc; k += 32) {
              const int f = k >> 2;
              const float v = eval_item32(g, RF, q, col0 + f, r, gm);
              if (r == 0) out[ob + f] = v;
            }
          }
        }
        if (MODE == MODE_MC && lane < ne) out[(e0 + lane) * (long long)per + 2 * g.nf] = RF.as[lane];
      }
      __syncwarp();
      continue;
    }

    // ---- phase 2, FP64, member sets: the same sites for every member ----
    if constexpr (MODE == MODE_MEMBERS) {
      const WarpRec<double> &RD = reinterpret_cast<const WarpRec<double> &>(R);
      const int m1 = min(g.nmem, (chunk + 1) * mchunk);
      for (int m = chunk * mchunk; m < m1; m++) {
        const size_t moff = (size_t)m * g.mstride;
        const int nitems = ne * per;
        int p = lane / per, c = lane - (lane / per) * per;
        for (int k = lane; k < nitems; k += 32) {
          out[((long long)m * n + e0 + RD.orig[p]) * per + c] = (T)eval_item64(g, RD, p, c, moff);
          c += dc;
          p += dp;
          if (c >= per) { c -= per; p++; }
        }
      }
      __syncwarp();
      continue;
    }

    // ---- phase 2, FP64: items = (point, column), one lane each ----
    const int nitems = ne * per;
    int p = (lane / LPI) / per, c = (lane / LPI) - ((lane / LPI) / per) * per;
    for (int k = lane / LPI; k < nitems; k += IPI) {
      T v;
      long long o;
      int pt, col;
      if (MODE == MODE_POINTS) {
        pt = p;
        col = col0 + c;
        o = (e0 + R.orig[p]) * (long long)per + c;
      } else {
        const int side = c >= g.nf;
        pt = 2 * p + side;
        col = c - side * g.nf;
        o = (e0 + p) * (long long)per + c;
      }
      if (MODE == MODE_MC && c == 2 * g.nf) {
        v = R.as[p];
      } else {
        v = (T)eval_item64(g, reinterpret_cast<const WarpRec<double> &>(R), pt, col);
      }
      out[o] = v;
      c += dc;
      p += dp;
      if (c >= per) { c -= per; p++; }
    }
    __syncwarp();
  }
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_alphas(GridView g, const T *__restrict__ qa,
                                                     long long n, T *__restrict__ out) {
  using K = typename Prec<T>::K;
  extern __shared__ __align__(16) unsigned char smem[];
  K *akeys = reinterpret_cast<K *>(smem);
  load_keys<T>(g, akeys, 2);
  __syncthreads();
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long base = (long long)blockIdx.x * blockDim.x; base < n; base += stride) {
    long long i = base + threadIdx.x;
    bool present = i < n;
    T q2 = present ? qa[i] : T(1);
    bool bad = present && !((q2 > T(0)) && (q2 < T(INFINITY)));
    unsigned inv = __ballot_sync(0xffffffffu, bad);
    if ((threadIdx.x & 31) == 0 && inv) atomicAdd(g.invalid, (unsigned long long)__popc(inv));
    if (present) out[i] = alphas_eval(g, akeys, q2);
  }
}

// ---------------------------------------------------------------------------
// launch helpers
// ---------------------------------------------------------------------------
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

template <typename T, int MODE>
static size_t xf_smem(const GridView &g) {
  using K = typename std::conditional<sizeof(T) == 8, long long, int>::type;
  return keys_bytes(g.nx, sizeof(K)) + keys_bytes(g.nrows, sizeof(K)) +
         (MODE == MODE_MC ? keys_bytes(g.na, sizeof(K)) : 0) + kWarps * sizeof(WarpRec<T>);
}

template <typename T, int MODE>
static int launch_xf(const pdf_grid *grid, const T *xa, const T *qa, const T *xb, T s,
                     long long n, int col0, int ncol, T *out, cudaStream_t st) {
  const GridView &g = grid->v;
  size_t smem = xf_smem<T, MODE>(g);
  auto kern = k_xf<T, MODE>;
  static int configured = 0;
  if (smem > 48 * 1024 || !configured) {
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    configured = 1;
  }
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem);
  if (per_sm < 1) per_sm = 1;
  const int per_tile = MODE == MODE_MC ? 16 : 32;
  long long ntiles = (n + per_tile - 1) / per_tile;
  long long cap = (long long)num_sms() * per_sm;
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
  kern<<<(unsigned)blocks, kThreads, smem, st>>>(g, xa, qa, xb, s, n, col0, ncol, mchunk, out);
  return check_launch(MODE == MODE_MC ? "pdf_mc_event kernel" : "xfxq2 kernel");
}

template <typename T>
static int launch_alphas(const pdf_grid *grid, const T *q2, long long n, T *out, cudaStream_t st) {
  const GridView &g = grid->v;
  using K = typename std::conditional<sizeof(T) == 8, long long, int>::type;
  size_t smem = keys_bytes(g.na, sizeof(K));
  long long blocks = (n + kThreads - 1) / kThreads;
  long long cap = (long long)num_sms() * 8;
  if (blocks > cap) blocks = cap;
  k_alphas<T><<<(unsigned)blocks, kThreads, smem, st>>>(g, q2, n, out);
  return check_launch("alphas_q2 kernel");
}

static int check_common(const pdf_grid *g, const void *a, const void *b, const void *o, size_t n,
                        const char *what) {
  if (!g) return set_error(PDF_ERR_NULL, "%s: grid is NULL", what);
  if (n > 0 && (!a || !b || !o)) return set_error(PDF_ERR_NULL, "%s: NULL array", what);
  if (n > (size_t)1 << 40) return set_error(PDF_ERR_ARG, "%s: n = %zu too large", what, n);
  return PDF_OK;
}

template <typename T>
static int do_xfxq2(const pdf_grid *g, int pid, const T *x, const T *q2, size_t n, T *out,
                    cudaStream_t st) {
  int rc = check_common(g, x, q2, out, n, "xfxq2");
  if (rc) return rc;
  int col = pdf_grid_pid_column(g, pid);
  if (col < 0) return set_error(PDF_ERR_PID, "xfxq2: pid %d not in the grid", pid);
  if (n == 0) return PDF_OK;
  return launch_xf<T, MODE_POINTS>(g, x, q2, nullptr, T(0), (long long)n, col, 1, out, st);
}

template <typename T>
static int do_all(const pdf_grid *g, const T *x, const T *q2, size_t n, T *out, cudaStream_t st) {
  int rc = check_common(g, x, q2, out, n, "xfxq2_all_flavours");
  if (rc) return rc;
  if (n == 0) return PDF_OK;
  return launch_xf<T, MODE_POINTS>(g, x, q2, nullptr, T(0), (long long)n, 0, g->v.nf, out, st);
}

template <typename T>
static int do_alphas(const pdf_grid *g, const T *q2, size_t n, T *out, cudaStream_t st) {
  int rc = check_common(g, q2, q2, out, n, "alphas_q2");
  if (rc) return rc;
  if (g->v.na == 0) return set_error(PDF_ERR_NO_ALPHAS, "alphas_q2: grid has no alpha_s nodes");
  if (n == 0) return PDF_OK;
  return launch_alphas<T>(g, q2, (long long)n, out, st);
}

template <typename T>
static int do_mc(const pdf_grid *g, const T *x1, const T *x2, T s, size_t n, T *out, cudaStream_t st) {
  int rc = check_common(g, x1, x2, out, n, "pdf_mc_event");
  if (rc) return rc;
  if (g->v.na == 0) return set_error(PDF_ERR_NO_ALPHAS, "pdf_mc_event: grid has no alpha_s nodes");
  if (!(s > T(0)) || !(s < T(INFINITY))) return set_error(PDF_ERR_ARG, "pdf_mc_event: s must be positive and finite");
  if (n == 0) return PDF_OK;
  return launch_xf<T, MODE_MC>(g, x1, nullptr, x2, s, (long long)n, 0, 0, out, st);
}

int launch_members_f64(const pdf_grid *g, const double *x, const double *q2, long long n, double *out,
                       cudaStream_t st) {
  return launch_xf<double, MODE_MEMBERS>(g, x, q2, nullptr, 0.0, n, 0, g->v.nf, out, st);
}

// Used by the host-memory path.
int launch_alphas_f64(const pdf_grid *g, const double *q2, long long n, double *out, cudaStream_t st) {
  return launch_alphas<double>(g, q2, n, out, st);
}
int launch_all_f64(const pdf_grid *g, const double *x, const double *q2, long long n, double *out,
                   cudaStream_t st) {
  return launch_xf<double, MODE_POINTS>(g, x, q2, nullptr, 0.0, n, 0, g->v.nf, out, st);
}

}  // namespace pdfgb

using namespace pdfgb;

extern "C" int xfxq2(const pdf_grid *g, int pid, const double *x, const double *q2, size_t n,
                     double *out, cudaStream_t st) {
  return do_xfxq2<double>(g, pid, x, q2, n, out, st);
}
extern "C" int xfxq2_f32(const pdf_grid *g, int pid, const float *x, const float *q2, size_t n,
                         float *out, cudaStream_t st) {
  return do_xfxq2<float>(g, pid, x, q2, n, out, st);
}
extern "C" int xfxq2_all_flavours(const pdf_grid *g, const double *x, const double *q2, size_t n,
                                  double *out, cudaStream_t st) {
  return do_all<double>(g, x, q2, n, out, st);
}
extern "C" int xfxq2_all_flavours_f32(const pdf_grid *g, const float *x, const float *q2, size_t n,
                                      float *out, cudaStream_t st) {
  return do_all<float>(g, x, q2, n, out, st);
}
extern "C" int alphas_q2(const pdf_grid *g, const double *q2, size_t n, double *out, cudaStream_t st) {
  return do_alphas<double>(g, q2, n, out, st);
}
extern "C" int alphas_q2_f32(const pdf_grid *g, const float *q2, size_t n, float *out, cudaStream_t st) {
  return do_alphas<float>(g, q2, n, out, st);
}
extern "C" int xfxq2_all_members(const pdf_grid *g, const double *x, const double *q2, size_t n, double *out,
                                 cudaStream_t st) {
  int rc = check_common(g, x, q2, out, n, "xfxq2_all_members");
  if (rc) return rc;
  if (n == 0) return PDF_OK;
  return launch_members_f64(g, x, q2, (long long)n, out, st);
}

extern "C" int pdf_mc_event(const pdf_grid *g, const double *x1, const double *x2, double s, size_t n,
                            double *out, cudaStream_t st) {
  return do_mc<double>(g, x1, x2, s, n, out, st);
}
extern "C" int pdf_mc_event_f32(const pdf_grid *g, const float *x1, const float *x2, float s, size_t n,
                                float *out, cudaStream_t st) {
  return do_mc<float>(g, x1, x2, s, n, out, st);
}
