// adjoint.cu -- vector-Jacobian product of xfxq2_all_flavours.
//
// For L = sum_p sum_f c[p][f] xf_f(x_p, Q^2_p) the kernel returns dL/dx_p,
// dL/dQ^2_p and accumulates dL/d(knot values).  One thread per point loops
// over the flavours: per flavour and patch site it evaluates the patch F and
// its derivatives F_t, F_u from the cell's Bezier control points, pushes them
// through the continuation rule of the point's class (chain rule), and
// scatters c * dxf/dF * w_a(t) w_b(u) into the knot-value gradient with FP64
// atomics, w_a the tangent-augmented Hermite weight of knot a (the patch is
// linear in the knot values: dF/df_ab = w_a(t) w_b(u)).  The x and Q^2
// derivatives are summed over flavours in registers, in a fixed order.
//
// A query exactly on the last x (or top Q^2) knot is taken in the last
// proper cell at t = 1 (u = 1), so the derivative there is the one-sided one
// of that cell.
#include "sites.cuh"

namespace pdfgb {

constexpr int kAdjThreads = 256;

struct Site64 {
  double B[4], dB[4];  // Bernstein weights and derivatives in the cell position
  double w[4];         // knot weights w_a(t) of the cell
  int c, k0;           // cell index (x: cell, q: Q cell) and first knot (col / row) of the stencil
  double dpos;         // d(position)/d(coordinate), 0 for a fixed site
};

__device__ __forceinline__ void bern_d(double t, double s, double *B, double *dB) {
  double t2 = t * t, s2 = s * s;
  B[0] = s2 * s; B[1] = 3.0 * t * s2; B[2] = 3.0 * t2 * s; B[3] = t2 * t;
  dB[0] = -3.0 * s2; dB[1] = 3.0 * s * (s - 2.0 * t); dB[2] = 3.0 * t * (2.0 * s - t); dB[3] = 3.0 * t2;
}

__device__ __forceinline__ void make_site(Site64 &S, const double *Wc, double t, double s, int cell, int k0,
                                          double dpos) {
  bern_d(t, s, S.B, S.dB);
  for (int a = 0; a < 4; a++)
    S.w[a] = Wc[a * 4] * S.B[0] + Wc[a * 4 + 1] * S.B[1] + Wc[a * 4 + 2] * S.B[2] + Wc[a * 4 + 3] * S.B[3];
  S.c = cell;
  S.k0 = k0;
  S.dpos = dpos;
}

// Patch value and its derivatives in t and u.
__device__ __forceinline__ void patch_d(const double *b, const Site64 &X, const Site64 &Q, double &F,
                                        double &Ft, double &Fu) {
  F = Ft = Fu = 0.0;
  for (int l = 0; l < 4; l++) {
    const double2 *q = reinterpret_cast<const double2 *>(b + 4 * l);
    double2 v0 = __ldg(q), v1 = __ldg(q + 1);
    double r = X.B[0] * v0.x + X.B[1] * v0.y + X.B[2] * v1.x + X.B[3] * v1.y;
    double rt = X.dB[0] * v0.x + X.dB[1] * v0.y + X.dB[2] * v1.x + X.dB[3] * v1.y;
    F = fma(Q.B[l], r, F);
    Ft = fma(Q.B[l], rt, Ft);
    Fu = fma(Q.dB[l], r, Fu);
  }
}

// Pair rule with its partial derivatives in g0, g1, p.
__device__ __forceinline__ double pair_d(double g0, double g1, double p, double &d0, double &d1, double &dp) {
  if (g0 > 0.0 && g1 > 0.0) {
    double lr = log(g1 / g0);
    double v = g0 * exp(p * lr);
    d0 = v * (1.0 - p) / g0;
    d1 = v * p / g1;
    dp = v * lr;
    return v;
  }
  d0 = 1.0 - p;
  d1 = p;
  dp = g1 - g0;
  return g0 + (g1 - g0) * p;
}

// Low-Q^2 rule with its partial derivatives in f0, f1, rho.
__device__ __forceinline__ double lowq_d(double f0, double f1, double rho, double lr, double L, double &d0,
                                         double &d1, double &drho) {
  bool pos = f0 > 0.0 && f1 > 0.0;
  double gam = pos ? log(f1 / f0) / L : 1.0;
  double ex = (gam * rho + 1.0) - rho;
  double e = exp(ex * lr);
  double v = f0 * e;
  d0 = pos ? e * (1.0 - lr * rho / L) : e;
  d1 = pos ? v * lr * rho / (f1 * L) : 0.0;
  drho = v * ((gam - 1.0) * lr + ex / rho);
  return v;
}

// The whole vector-Jacobian product of one point: d/dx, d/dQ^2 into gx[p],
// gq[p], knot-value contributions added to gv.
__device__ __forceinline__ void vjp_point(const GridView &g, const long long *xkeys, const long long *qkeys,
                                          long long p, const double *__restrict__ xa,
                                          const double *__restrict__ qa, const double *__restrict__ cot,
                                          double *__restrict__ gx, double *__restrict__ gq,
                                          double *__restrict__ gv) {
    const double x = xa[p], q2 = qa[p];
    double lq;
    PointSites<double> ps = sites(g, xkeys, qkeys, x, q2, LogTabs{g.tlogtab, g.tloghtab}, lq);
    if (ps.cls == C_INVALID) {
      if (gx) gx[p] = NAN;
      if (gq) gq[p] = NAN;
      return;
    }
    const bool lowx = ps.cls == C_LOWX || ps.cls == C_LOWX_HIGHQ || ps.cls == C_LOWX_LOWQ;
    const bool realq = ps.cls == C_IN || ps.cls == C_LOWX;
    // a query on the last knot: derivative of the last proper cell at t = 1
    if (!lowx && ps.xc0 == g.nx - 1) { ps.xc0 = g.nx - 2; ps.t0 = 1.0; ps.ts0 = 0.0; }
    if (realq && ps.qc0 == g.nqc) { ps.qc0 = g.top_qc; ps.u0 = 1.0; ps.us0 = 0.0; }
    Site64 X[2], Q[2];
    for (int a = 0; a < 2; a++) {
      int xc = a ? ps.xc1 : ps.xc0;
      double t = a ? ps.t1 : ps.t0, s = a ? 1.0 - ps.t1 : ps.ts0;
      double dpos = (a == 0 && !lowx) ? g.xcell[4 * xc + 1] / x : 0.0;
      make_site(X[a], g.xW + 16 * xc, t, s, xc, xc - 1, dpos);
    }
    for (int b = 0; b < 2; b++) {
      int qc = b ? ps.qc1 : ps.qc0;
      double u = b ? ps.u1 : ps.u0, s = b ? 1.0 - ps.u1 : ps.us0;
      int row = g.qc_row[qc];
      double dpos = (b == 0 && realq) ? g.qcell[4 * row + 1] / q2 : 0.0;
      make_site(Q[b], g.qW + 16 * qc, u, s, qc, row - 1, dpos);
    }
    const int nsx = lowx ? 2 : 1;
    const int nsq = (ps.cls == C_IN || ps.cls == C_LOWX) ? 1 : 2;
    const double dpx = lowx ? g.idx0 / x : 0.0;
    const double dpq = (ps.cls == C_HIGHQ || ps.cls == C_LOWX_HIGHQ) ? -g.idq_top / q2 : 0.0;
    const double drho = (ps.cls == C_LOWQ || ps.cls == C_LOWX_LOWQ) ? 1.0 / g.q2min : 0.0;
    double sx = 0.0, sq = 0.0;
    for (int f = 0; f < g.nf; f++) {
      const double c = cot[p * g.nf + f];
      double F[2][2], Ft[2][2], Fu[2][2];
      for (int a = 0; a < nsx; a++)
        for (int b = 0; b < nsq; b++) {
          const double *blk = g.coef + (((size_t)Q[b].c * g.nx + X[a].c) * g.nf + f) * 16;
          patch_d(blk, X[a], Q[b], F[a][b], Ft[a][b], Fu[a][b]);
        }
      double lam[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
      double dvpx = 0.0, dvpq = 0.0, dvrho = 0.0, d0, d1, dp;
      switch (ps.cls) {
        case C_IN: lam[0][0] = 1.0; break;
        case C_LOWX: pair_d(F[0][0], F[1][0], ps.px, lam[0][0], lam[1][0], dvpx); break;
        case C_HIGHQ: pair_d(F[0][0], F[0][1], ps.pq, lam[0][0], lam[0][1], dvpq); break;
        case C_LOWQ: lowq_d(F[0][0], F[0][1], ps.pq, ps.lr, g.ln101, lam[0][0], lam[0][1], dvrho); break;
        case C_LOWX_HIGHQ: {
          double a0, a1, ap, b0, b1, bp;
          double A = pair_d(F[0][0], F[0][1], ps.pq, a0, a1, ap);
          double B = pair_d(F[1][0], F[1][1], ps.pq, b0, b1, bp);
          pair_d(A, B, ps.px, d0, d1, dp);
          lam[0][0] = d0 * a0; lam[0][1] = d0 * a1; lam[1][0] = d1 * b0; lam[1][1] = d1 * b1;
          dvpq = d0 * ap + d1 * bp;
          dvpx = dp;
          break;
        }
        case C_LOWX_LOWQ: {
          double a0, a1, ar, b0, b1, br;
          double A = lowq_d(F[0][0], F[0][1], ps.pq, ps.lr, g.ln101, a0, a1, ar);
          double B = lowq_d(F[1][0], F[1][1], ps.pq, ps.lr, g.ln101, b0, b1, br);
          pair_d(A, B, ps.px, d0, d1, dp);
          lam[0][0] = d0 * a0; lam[0][1] = d0 * a1; lam[1][0] = d1 * b0; lam[1][1] = d1 * b1;
          dvrho = d0 * ar + d1 * br;
          dvpx = dp;
          break;
        }
      }
      double dx = dvpx * dpx, dq = dvpq * dpq + dvrho * drho;
      for (int a = 0; a < nsx; a++)
        for (int b = 0; b < nsq; b++) {
          dx = fma(lam[a][b] * Ft[a][b], X[a].dpos, dx);
          dq = fma(lam[a][b] * Fu[a][b], Q[b].dpos, dq);
          if (gv) {
            // zero tests on bit patterns (the FP64 pipe is the busy unit);
            // c lam w_b folded once per row, then times each w_a
            const double m = c * lam[a][b];
            if ((__double_as_longlong(m) << 1) == 0) continue;
            for (int bb = 0; bb < 4; bb++) {
              const int row = Q[b].k0 + bb;
              const double wq = Q[b].w[bb];
              if ((__double_as_longlong(wq) << 1) == 0 || row < 0 || row >= g.nrows) continue;
              const double mq = m * wq;
              for (int aa = 0; aa < 4; aa++) {
                const int col = X[a].k0 + aa;
                const double wx = X[a].w[aa];
                if ((__double_as_longlong(wx) << 1) == 0 || col < 0 || col >= g.nx) continue;
                atomicAdd(gv + ((size_t)row * g.nx + col) * g.nf + f, mq * wx);
              }
            }
          }
        }
      sx = fma(c, dx, sx);
      sq = fma(c, dq, sq);
    }
    if (gx) gx[p] = sx;
    if (gq) gq[p] = sq;
}

// One warp per tile of 32 points, a lane per point.  Points that need a
// continuation rule (found by integer range tests on the raw inputs) are
// queued per warp and processed 32 at a time, so that a warp of in-grid
// points never runs the continuation code (log, exp, division, four sites)
// for a few lanes -- the FP64 pipe would pay for all 32.
constexpr int kAdjWarps = kAdjThreads / 32;

__global__ void __launch_bounds__(kAdjThreads, 1)
k_vjp(GridView g, const double *__restrict__ xa, const double *__restrict__ qa, const double *__restrict__ cot,
      long long n, double *__restrict__ gx, double *__restrict__ gq, double *__restrict__ gv) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ long long queue[kAdjWarps][64];
  long long *xkeys = reinterpret_cast<long long *>(smem);
  long long *qkeys = reinterpret_cast<long long *>(smem + keys_bytes(g.nx, 8));
  load_keys<double>(g, xkeys, 0);
  load_keys<double>(g, qkeys, 1);
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  long long *Q = queue[warp];
  const unsigned lt = (1u << lane) - 1u;
  const long long kxlast = __double_as_longlong(g.xlast), kx0 = __double_as_longlong(g.x0);
  const long long kqmin = __double_as_longlong(g.q2min), kqmax = __double_as_longlong(g.q2max);
  int nq = 0;  // queued points (warp-uniform)
  const long long ntiles = (n + 31) / 32, nwarps = (long long)gridDim.x * kAdjWarps;
  long long tile = (long long)blockIdx.x * kAdjWarps + warp;
  // one call site: each round either drains 32 queued points, or takes the
  // in-grid points of the next tile (queueing its continuation points), or
  // drains the rest of the queue at the end (every branch is warp-uniform)
  while (true) {
    long long pp = -1;
    if (nq >= 32) {
      nq -= 32;
      pp = Q[nq + lane];
    } else if (tile < ntiles) {
      const long long p = tile * 32 + lane;
      bool far = false;
      if (p < n) {
        const long long kx = __double_as_longlong(xa[p]), kq = __double_as_longlong(qa[p]);
        const bool valid = kq > 0 && kq < 0x7FF0000000000000LL && kx > 0 && kx <= kxlast;
        far = valid && (kx < kx0 || kq < kqmin || kq > kqmax);
        if (!far) pp = p;
      }
      const unsigned fm = __ballot_sync(0xffffffffu, far);
      if (far) Q[nq + __popc(fm & lt)] = p;
      nq += __popc(fm);
      tile += nwarps;
    } else if (nq > 0) {
      if (lane < nq) pp = Q[lane];
      nq = 0;
    } else {
      break;
    }
    __syncwarp();
    if (pp >= 0) vjp_point(g, xkeys, qkeys, pp, xa, qa, cot, gx, gq, gv);
    __syncwarp();
  }
}

}  // namespace pdfgb

using namespace pdfgb;

extern "C" int xfxq2_all_flavours_vjp(const pdf_grid *grid, const double *x, const double *q2, size_t n,
                                      const double *cot, double *grad_x, double *grad_q2, double *grad_values,
                                      cudaStream_t stream) {
  if (!grid) return set_error(PDF_ERR_NULL, "xfxq2_all_flavours_vjp: grid is NULL");
  if (n > 0 && (!x || !q2 || !cot)) return set_error(PDF_ERR_NULL, "xfxq2_all_flavours_vjp: NULL array");
  if (n == 0) return PDF_OK;
  const GridView &g = grid->v;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  size_t smem = keys_bytes(g.nx, 8) + keys_bytes(g.nrows, 8);
  long long blocks = ((long long)n + kAdjThreads - 1) / kAdjThreads;  // one tile per warp at most
  long long cap = (long long)(sms > 0 ? sms : 1) * 8;
  if (blocks > cap) blocks = cap;
  k_vjp<<<(unsigned)blocks, kAdjThreads, smem, stream>>>(g, x, q2, cot, (long long)n, grad_x, grad_q2,
                                                         grad_values);
  return check_launch("xfxq2_all_flavours_vjp kernel");
}
