// adjoint.cu -- vector-Jacobian product of xfxq2_all_flavours.
//
// For L = sum_p sum_f c[p][f] xf_f(x_p, Q^2_p) the kernel returns dL/dx_p,
// dL/dQ^2_p and accumulates dL/d(knot values).  One lane per point loops
// over the flavours: per flavour and patch site it evaluates the patch F and
// its derivatives F_t, F_u from the cell's Bezier control points (in
// float-float for in-grid points, FP64 otherwise), pushes them through the
// continuation rule of the point's class (chain rule), and scatters
// c * dxf/dF * w_a(t) w_b(u) into the knot-value gradient with FP64 atomics,
// w_a the tangent-augmented Hermite weight of knot a (the patch is linear in
// the knot values: dF/df_ab = w_a(t) w_b(u)).  The x and Q^2 derivatives are
// summed over flavours in registers, in a fixed order.  Small batches run
// k_vjp (continuation points queued per warp by kind); batches of 2048
// points or more are first sorted by cell and run k_vjp_sorted, which
// contracts the knot-value terms of same-cell runs before its atomics.
//
// A query exactly on the last x (or top Q^2) knot is taken in the last
// proper cell at t = 1 (u = 1), so the derivative there is the one-sided one
// of that cell.
#include <algorithm>
#include <mutex>

#include "ff.cuh"
#include "ffsplit.cuh"
#include "sites.cuh"

namespace pdfgb {

constexpr int kAdjThreads = 256;

struct Site64 {
  double B[4], dB[4];  // Bernstein weights and derivatives in the cell position
  double w[4];         // knot weights w_a(t) of the cell
  int c, k0;           // cell index (x: cell, q: Q cell) and first knot (col / row) of the stencil
  double dpos;         // d(position)/d(coordinate), 0 for a fixed site
};


// A double as a float pair: split on the integer pipe within 2^+-50, else
// by FP64 conversions.
__device__ __forceinline__ ff2 ff_pair(double v) { return ff_safe(v, 50) ? ff_split50(v) : ff_of(v); }

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

// Patch value and its derivatives in t (when the x site moves with x) and u.
__device__ __forceinline__ void patch_d(const double *b, const Site64 &X, const Site64 &Q, bool need_t, double &F,
                                        double &Ft, double &Fu) {
  F = Ft = Fu = 0.0;
  for (int l = 0; l < 4; l++) {
    const double2 *q = reinterpret_cast<const double2 *>(b + 4 * l);
    double2 v0 = __ldg(q), v1 = __ldg(q + 1);
    double r = X.B[0] * v0.x + X.B[1] * v0.y + X.B[2] * v1.x + X.B[3] * v1.y;
    F = fma(Q.B[l], r, F);
    Fu = fma(Q.dB[l], r, Fu);
    if (need_t) {
      double rt = X.dB[0] * v0.x + X.dB[1] * v0.y + X.dB[2] * v1.x + X.dB[3] * v1.y;
      Ft = fma(Q.B[l], rt, Ft);
    }
  }
}

// The same for a site whose Bernstein weights in x (xk) or in u (qk) are
// (1, 0, 0, 0) -- a site on a knot, as the continuation rules' fixed sites
// are: only the first control point of each row, or the first row, enters,
// and the sums are exactly those of patch_d.  F_u only where the Q site
// moves with Q^2 (need_u); a fixed site's F_u would be multiplied by 0.
__device__ __forceinline__ void patch_site(const double *b, const Site64 &X, const Site64 &Q, bool xk, bool qk,
                                           bool need_t, bool need_u, double &F, double &Ft, double &Fu) {
  if (xk && !need_t) {
    F = Ft = Fu = 0.0;
#pragma unroll
    for (int l = 0; l < 4; l++) {
      const double v = __ldg(b + 4 * l);
      F = fma(Q.B[l], v, F);
      if (need_u) Fu = fma(Q.dB[l], v, Fu);
    }
    return;
  }
  if (qk && !need_u) {
    const double2 *q = reinterpret_cast<const double2 *>(b);
    const double2 v0 = __ldg(q), v1 = __ldg(q + 1);
    F = X.B[0] * v0.x + X.B[1] * v0.y + X.B[2] * v1.x + X.B[3] * v1.y;
    Ft = need_t ? X.dB[0] * v0.x + X.dB[1] * v0.y + X.dB[2] * v1.x + X.dB[3] * v1.y : 0.0;
    Fu = 0.0;
    return;
  }
  patch_d(b, X, Q, need_t, F, Ft, Fu);
}

// A continuation rule and its partial derivatives.  Both rules are of the
// log form v = f0 exp(a ln(f1/f0) + b): the pair rule with a = p, b = 0 (and
// v = f0 + (f1 - f0) p when f0 or f1 is not positive), the low-Q^2 rule with
// a = rho lr / ln1.01, b = (1 - rho) lr (a = 0, b = lr when f0 or f1 is not
// positive: gamma = 1).  Then dv/df0 = e (1 - a), dv/df1 = e a / r with
// e = exp(a ln r + b), r = f1/f0, and dv/dpar = dv/da da/dpar + dv/db db/dpar
// for the rule's parameter (p, or rho with lr = ln rho).  The same
// table-driven logarithm, exponential and reciprocal as the evaluation.
struct RuleD {
  double v, d0, d1, dpar;
};
__device__ __forceinline__ RuleD rule_d(double f0, double f1, double p, bool lowq, double rho, double lr,
                                        double irho, double iL, LogTabs LT, const double *ET) {
  RuleD R;
  const bool pos = __double_as_longlong(f0) > 0 && __double_as_longlong(f1) > 0;
  double r = 1.0, lnr = 0.0;
  if (pos) {
    r = ddiv(f1, f0);
    lnr = tlog(r, LT);
  }
  double a = p, b = 0.0;
  if (lowq) {
    a = pos ? rho * lr * iL : 0.0;
    b = pos ? (1.0 - rho) * lr : lr;
  }
  if (pos || lowq) {
    const double e = texp(fma(a, lnr, b), ET);
    R.v = f0 * e;
    R.d0 = e * (1.0 - a);
    R.d1 = pos ? ddiv(e * a, r) : 0.0;
    const double da = R.v * lnr, db = R.v;
    R.dpar = !lowq ? da : pos ? da * (lr + 1.0) * iL + db * ((1.0 - rho) * irho - lr) : db * irho;
  } else {
    R.v = f0 + (f1 - f0) * p;
    R.d0 = 1.0 - p;
    R.d1 = p;
    R.dpar = f1 - f0;
  }
  return R;
}

__device__ __noinline__ RuleD rule_d_fp64(double f0, double f1, double p, bool lowq, double rho, double lr,
                                          double irho, double iL, LogTabs LT, const double *ET) {
  return rule_d(f0, f1, p, lowq, rho, lr, irho, iL, LT, ET);
}

// The same rule in float-float on the FMA pipe (ffmath.cuh), for positive
// f0, f1 on a float-float-safe grid: the FP64 pipe keeps only the
// conversions in and out.  A rule's point constants as float pairs, once per
// point: a, b and 1 - a of the log form, and dv/dpar = v (k1 ln r + k2) --
// the pair rule k1 = 1, k2 = 0; the low-Q^2 rule k1 = (lr + 1) / ln1.01,
// k2 = (1 - rho) / rho - lr.  Anything outside the pairs' range (a quotient,
// exponent or result beyond 2^+-100, |exponent| >= 64), and f0 or f1 not
// positive, takes the FP64 rule.
struct RuleFF {
  ff2 a, b, oma, k1, k2;
  double p, rho, lr, irho, iL;
  bool lowq;
};
__device__ __forceinline__ RuleFF rule_ff_consts(double p, bool lowq, double rho, double lr, double irho,
                                                 double iL) {
  RuleFF c;
  c.p = p; c.rho = rho; c.lr = lr; c.irho = irho; c.iL = iL; c.lowq = lowq;
  // (explicit roundings: both kernels that inline this get the same constants)
  const double a = lowq ? __dmul_rn(__dmul_rn(rho, lr), iL) : p;
  c.a = ff_of(a);
  c.b = ff_of(lowq ? __dmul_rn(__dsub_rn(1.0, rho), lr) : 0.0);
  c.oma = ff_of(__dsub_rn(1.0, a));
  c.k1 = lowq ? ff_of(__dmul_rn(__dadd_rn(lr, 1.0), iL)) : ff2{1.f, 0.f};
  c.k2 = ff_of(lowq ? __dsub_rn(__dmul_rn(__dsub_rn(1.0, rho), irho), lr) : 0.0);
  return c;
}
__device__ __forceinline__ bool ff_fine(ff2 v) { return v.h == 0.f || (fabsf(v.h) >= 0x1p-100f && fabsf(v.h) < 0x1p100f); }
__device__ __forceinline__ RuleD rule_d_ff(double f0, double f1, const RuleFF &c, FFTabs FT, LogTabs LT,
                                           const double *ET) {
  if (__double_as_longlong(f0) > 0 && __double_as_longlong(f1) > 0) {
    const ff2 F0 = ff_of(f0), F1 = ff_of(f1);
    if (ff_fine(F0) && ff_fine(F1)) {
      const ff2 r = ff_div(F1, F0);
      if (ff_fine(r)) {
        const ff2 lnr = ff_log(r, FT);
        const ff2 y = ff_add(ff_mul(c.a, lnr), c.b);
        if (fabsf(y.h) < 64.f) {
          const ff2 e = ff_exp(y, FT);
          const ff2 v = ff_mul(F0, e);
          const ff2 d0 = ff_mul(e, c.oma);
          const ff2 d1 = ff_div(ff_mul(e, c.a), r);
          const ff2 dp = ff_mul(v, ff_add(ff_mul(c.k1, lnr), c.k2));
          if (ff_fine(v) && ff_fine(d0) && ff_fine(d1) && ff_fine(dp))
            return {ff_to_d(v), ff_to_d(d0), ff_to_d(d1), ff_to_d(dp)};
        }
      }
    }
  }
  return rule_d_fp64(f0, f1, c.p, c.lowq, c.rho, c.lr, c.irho, c.iL, LT, ET);
}

// Where an in-grid point leaves its knot-weight terms for the warp's
// contraction (k_vjp_sorted): its 16 weights w_b(u) w_a(t) and its nf
// cotangents as float-float pairs, its cell and the cell's first knot.
struct Staged {
  float2 *w, *c;
  int cell, xk0, qk0;
  bool ing;
  double *gvc;  // where a continuation point's knot terms go (one of the private copies, or gv)
};

// FP64 knot scatter of one in-grid point, out of line: the staged path
// takes it only for a point whose weights or cotangents are too small or
// large for float-float (rare), and keeps its registers off the hot path.
__device__ __noinline__ void scatter_point_f64(int nrows, int nx, int nf, double wq0, double wq1, double wq2,
                                               double wq3, double wx0, double wx1, double wx2, double wx3,
                                               int qk0, int xk0, const double *__restrict__ cp,
                                               double *__restrict__ gv) {
  const double wq[4] = {wq0, wq1, wq2, wq3}, wx[4] = {wx0, wx1, wx2, wx3};
  for (int f = 0; f < nf; f++) {
    const double c = cp[f];
    if ((__double_as_longlong(c) << 1) == 0) continue;
    for (int m = 0; m < 16; m++) {
      const int row = qk0 + (m >> 2), col = xk0 + (m & 3);
      const double w = wq[m >> 2] * wx[m & 3];
      if (row >= 0 && row < nrows && col >= 0 && col < nx && (__double_as_longlong(w) << 1) != 0)
        atomicAdd(gv + ((size_t)row * nx + col) * nf + f, c * w);
    }
  }
}

// Bernstein weights and their t-derivatives in float-float from the site's
// position t and its complement s (computed apart, so whichever is small
// keeps its precision): four conversions on the FP64 pipe, the rest on the
// FMA pipe.  dB/dt = (-3 s^2, 3 s^2 - 6 t s, 6 t s - 3 t^2, 3 t^2).
// (ff_sub: ffmath.cuh)
__device__ __forceinline__ void ff_bern_d(double t, double s, ff2 dpos, ff2 *B, ff2 *dB) {
  const ff2 tf = ff_pair(t), sf = ff_pair(s), three = {3.f, 0.f}, six = {6.f, 0.f};
  const ff2 t2 = ff_mul(tf, tf), s2 = ff_mul(sf, sf), ts = ff_mul(tf, sf);
  B[0] = ff_mul(s2, sf);
  B[1] = ff_mul(three, ff_mul(tf, s2));
  B[2] = ff_mul(three, ff_mul(t2, sf));
  B[3] = ff_mul(t2, tf);
  const ff2 s23 = ff_mul(three, s2), t23 = ff_mul(three, t2), ts6 = ff_mul(six, ts);
  dB[0] = ff_mul(ff2{-s23.h, -s23.l}, dpos);
  dB[1] = ff_mul(ff_sub(s23, ts6), dpos);
  dB[2] = ff_mul(ff_sub(ts6, t23), dpos);
  dB[3] = ff_mul(t23, dpos);
}

// The knot weights w_a = sum_k W[a][k] B_k of a proper cell (the Hermite
// weights of the cell tables, grid.cu: W[1][0] = W[2][3] = 1, and besides
// those only W[0][1], W[1][1], W[1][2], W[2][1], W[2][2], W[3][2] nonzero)
// in float-float from the float-float Bernstein basis B.  false if an entry
// is outside 2^+-50 (then the caller takes the FP64 weights).
__device__ __forceinline__ bool ff_knot_weights(const double *Wc, const ff2 *B, ff2 *w) {
  const double e01 = Wc[1], e11 = Wc[5], e12 = Wc[6], e21 = Wc[9], e22 = Wc[10], e32 = Wc[14];
  if (!(ff_safe(e01, 50) && ff_safe(e11, 50) && ff_safe(e12, 50) && ff_safe(e21, 50) && ff_safe(e22, 50) &&
        ff_safe(e32, 50)))
    return false;
  w[0] = ff_mul(ff_split50(e01), B[1]);
  w[1] = ff_add(ff_add(B[0], ff_mul(ff_split50(e11), B[1])), ff_mul(ff_split50(e12), B[2]));
  w[2] = ff_add(ff_add(ff_mul(ff_split50(e21), B[1]), ff_mul(ff_split50(e22), B[2])), B[3]);
  w[3] = ff_mul(ff_split50(e32), B[2]);
  return true;
}
// FP64 knot weights of both sites and their float pairs (out of line: the
// rare case of a cell table entry outside the pairs' range).
__device__ __noinline__ void site_weights_f64(const double *Wx, const double *Wq, double t, double ts, double u,
                                              double us, double *xw, double *qw, ff2 *wxf, ff2 *wqf) {
  Site64 Xf, Qf;
  make_site(Xf, Wx, t, ts, 0, 0, 0.0);
  make_site(Qf, Wq, u, us, 0, 0, 0.0);
  for (int k = 0; k < 4; k++) {
    xw[k] = Xf.w[k];
    qw[k] = Qf.w[k];
    wxf[k] = ff_of(xw[k]);
    wqf[k] = ff_of(qw[k]);
  }
}
// 0, or 2^-lim <= |v| < 2^lim, for a float pair
__device__ __forceinline__ bool ff_safe_pair(ff2 v, int lim) {
  const float a = fabsf(v.h);
  return a == 0.f || (a >= __uint_as_float((unsigned)(127 - lim) << 23) && a < __uint_as_float((unsigned)(127 + lim) << 23));
}

// ---- in-grid points on a float-float-safe grid ------------------------------
// An in-grid point: F_t dt/dx = sum_lk B_l(u) B'_k(t) dt/dx c_lk and F_u du/dQ^2
// (likewise) for every flavour in float-float on the FMA pipe from the
// float-float control points (good to ~2^-46 of sum |w c|); the coordinate
// sums in float-float with the knot gradient (else FP64).  The knot scatter
// (the patch is linear in the knot values with weights w_a(t) w_b(u)): FP64
// products and atomics per point, or (STAGE) the weights and cotangents
// staged for the warp's contraction.
template <bool STAGE>
__device__ __forceinline__ void vjp_ingrid_ff(const GridView &g, const Site64 &X, const Site64 &Q, ff2 dposx,
                                              ff2 dposq, double t, double ts, double u, double us, long long p,
                                              const double *__restrict__ cot, double *__restrict__ gx,
                                              double *__restrict__ gq, double *__restrict__ gv, Staged *st) {
  ff2 wt[16], wu[16];
  // the knot weights in float-float (the sorted kernel with the knot
  // gradient: from the Bernstein basis below; FP64 weights, out of line in
  // site_weights_f64, only where a cell table entry is out of range; the
  // sorted kernel's sites carry no FP64 weights, the per-point kernel's do)
  ff2 wxf[4], wqf[4];
  bool wff = false;
  {
    ff2 xb[4], xd[4], qb[4], qd[4];
    ff_bern_d(t, ts, dposx, xb, xd);
    ff_bern_d(u, us, dposq, qb, qd);
#pragma unroll
    for (int m = 0; m < 16; m++) {
      wt[m] = ff_mul(qb[m >> 2], xd[m & 3]);
      wu[m] = ff_mul(qd[m >> 2], xb[m & 3]);
    }
    if (STAGE && gv)
      wff = ff_knot_weights(g.xW + 16 * X.c, xb, wxf) && ff_knot_weights(g.qW + 16 * Q.c, qb, wqf);
  }
  double xw64[4], qw64[4];  // FP64 knot weights (a table entry out of the pairs' range)
  if (STAGE && gv && !wff) site_weights_f64(g.xW + 16 * X.c, g.qW + 16 * Q.c, t, ts, u, us, xw64, qw64, wxf, wqf);
  // staged only when every weight and cotangent is 0 or of moderate size, so
  // that each knot's float-float sum keeps its precision relative to that
  // knot's own terms; otherwise this point scatters in FP64
  // (the cotangents are checked as the flavour loop reads them)
  bool stage = false;
  if (STAGE && gv) {
    stage = true;
#pragma unroll
    for (int k = 0; k < 4; k++) stage = stage && ff_safe_pair(wqf[k], 25) && ff_safe_pair(wxf[k], 25);
  }
  double W[16];  // knot weights w_b(u) w_a(t), 0 where the knot is outside the grid
  if (!STAGE) {
#pragma unroll
    for (int m = 0; m < 16; m++) {
      const int row = Q.k0 + (m >> 2), col = X.k0 + (m & 3);
      W[m] = (row >= 0 && row < g.nrows && col >= 0 && col < g.nx) ? Q.w[m >> 2] * X.w[m & 3] : 0.0;
    }
  } else if (stage) {
#pragma unroll
    for (int m = 0; m < 16; m++) {
      const ff2 w = ff_mul(wqf[m >> 2], wxf[m & 3]);
      st->w[m] = make_float2(w.h, w.l);
    }
    st->cell = Q.c * g.nx + X.c;
    st->xk0 = X.k0;
    st->qk0 = Q.k0;
    st->ing = true;
  }
  const float4 *cb = reinterpret_cast<const float4 *>(g.coefff + ((size_t)Q.c * g.nx + X.c) * 16 * g.nfp);
  const long long k0 = ((long long)Q.k0 * g.nx + X.k0) * g.nf;  // knot (Q.k0, X.k0); the used ones are >= 0
  // the coordinate sums sum_f c_f F_t,f and sum_f c_f F_u,f: with the knot
  // gradient, in float-float for the flavours whose cotangent is of moderate
  // size (its float pair is needed for the staging anyway), else in FP64
  double sx = 0.0, sq = 0.0;
  ff2 sxf = {0.f, 0.f}, sqf = {0.f, 0.f};
  for (int f = 0; f < g.nf; f++) {
    const double c = cot[p * g.nf + f];
    float th = 0.f, tl = 0.f, uh = 0.f, ul = 0.f;
#pragma unroll
    for (int m2 = 0; m2 < 8; m2++) {
      const float4 b = __ldg(cb + (size_t)m2 * g.nfp + f);
      // b = {hi_m, hi_m+1, lo_m, lo_m+1}, m = 2 m2
      ff_acc(th, tl, wt[2 * m2], b.x, b.z);
      ff_acc(uh, ul, wu[2 * m2], b.x, b.z);
      ff_acc(th, tl, wt[2 * m2 + 1], b.y, b.w);
      ff_acc(uh, ul, wu[2 * m2 + 1], b.y, b.w);
    }
    const bool cmod = gv && ff_safe(c, 50);
    const ff2 cf = cmod ? ff_split50(c) : ff2{0.f, 0.f};
    if (cmod) {
      sxf = ff_add(sxf, ff_mul(cf, ff_two_sum(th, tl)));
      sqf = ff_add(sqf, ff_mul(cf, ff_two_sum(uh, ul)));
    } else {
      sx = fma(c, f2d(th) + f2d(tl), sx);
      sq = fma(c, f2d(uh) + f2d(ul), sq);
    }
    if (STAGE) {
      if (stage) {
        stage = cmod;
        float *cp = reinterpret_cast<float *>(st->c) + 4 * (f >> 1) + (f & 1);  // pair f / 2: {hi, hi, lo, lo}
        cp[0] = cf.h;
        cp[2] = cf.l;
      }
    } else if (gv && (__double_as_longlong(c) << 1) != 0) {
#pragma unroll
      for (int m = 0; m < 16; m++)
        if ((__double_as_longlong(W[m]) << 1) != 0)
          atomicAdd(gv + (k0 + ((long long)(m >> 2) * g.nx + (m & 3)) * g.nf + f), c * W[m]);
    }
  }
  if (STAGE && gv && !stage) {  // not staged after all: FP64 scatter instead
    st->ing = false;
    if (wff)
      scatter_point_f64(g.nrows, g.nx, g.nf, ff_to_d(wqf[0]), ff_to_d(wqf[1]), ff_to_d(wqf[2]), ff_to_d(wqf[3]),
                        ff_to_d(wxf[0]), ff_to_d(wxf[1]), ff_to_d(wxf[2]), ff_to_d(wxf[3]), Q.k0, X.k0,
                        cot + p * g.nf, gv);
    else
      scatter_point_f64(g.nrows, g.nx, g.nf, qw64[0], qw64[1], qw64[2], qw64[3], xw64[0], xw64[1], xw64[2],
                        xw64[3], Q.k0, X.k0, cot + p * g.nf, gv);
  }
  if (STAGE && stage)  // the pairs' unused flavours (up to 16) contract as zeros
    for (int f = g.nf; f < 16; f++) {
      float *cp = reinterpret_cast<float *>(st->c) + 4 * (f >> 1) + (f & 1);
      cp[0] = 0.f;
      cp[2] = 0.f;
    }
  sx += ff_to_d(sxf);
  sq += ff_to_d(sqf);
  if (gx) gx[p] = sx;
  if (gq) gq[p] = sq;
}

// The whole vector-Jacobian product of one point: d/dx, d/dQ^2 into gx[p],
// gq[p], knot-value contributions added to gv (an in-grid point's staged
// for the warp's contraction instead, with STAGE).
template <bool STAGE>
__device__ __forceinline__ void vjp_point(const GridView &g, const long long *xkeys, const long long *qkeys,
                                          LogTabs LT, const double *ET, long long p, const double *__restrict__ xa,
                                          const double *__restrict__ qa, const double *__restrict__ cot,
                                          double *__restrict__ gx, double *__restrict__ gq,
                                          double *__restrict__ gv, Staged *st) {
    const double x = xa[p], q2 = qa[p];
    double lq;
    PointSites<double> ps = g.ffpos ? sites_ffpos(g, xkeys, qkeys, g.lnfff, g.lnfff2, x, q2, LT, lq)
                                    : sites(g, xkeys, qkeys, x, q2, LT, lq);
    if (ps.cls == C_INVALID) {
      if (gx) gx[p] = NAN;
      if (gq) gq[p] = NAN;
      return;
    }
    const int cls = ps.cls;
    const bool lowx = cls == C_LOWX || cls == C_LOWX_HIGHQ || cls == C_LOWX_LOWQ;
    const bool realq = cls == C_IN || cls == C_LOWX;
    const bool lowq = cls == C_LOWQ || cls == C_LOWX_LOWQ;
    // a query on the last knot: derivative of the last proper cell at t = 1
    if (!lowx && ps.xc0 == g.nx - 1) { ps.xc0 = g.nx - 2; ps.t0 = 1.0; ps.ts0 = 0.0; }
    if (realq && ps.qc0 == g.nqc) { ps.qc0 = g.top_qc; ps.u0 = 1.0; ps.us0 = 0.0; }
    if (STAGE && cls == C_IN && g.ff) {
      // the sorted kernel's in-grid point: its sites' cells and first knots,
      // and d(position)/d(coordinate) = (1 / cell width) / coordinate as float
      // pairs; the Bernstein and knot weights are taken in float-float by
      // vjp_ingrid_ff
      Site64 Xs, Qs;
      Xs.c = ps.xc0;
      Xs.k0 = ps.xc0 - 1;
      const int row = g.qc_row[ps.qc0];
      Qs.c = ps.qc0;
      Qs.k0 = row - 1;
      const double idx = g.xcell[4 * ps.xc0 + 1], idq = g.qcell[4 * row + 1];
      ff2 dpx, dpq;
      if (ff_safe(x, 50) && ff_safe(q2, 50) && ff_safe(idx, 50) && ff_safe(idq, 50)) {
        dpx = ff_div(ff_split50(idx), ff_split50(x));
        dpq = ff_div(ff_split50(idq), ff_split50(q2));
      } else {
        dpx = ff_of(idx * ddiv(1.0, x));
        dpq = ff_of(idq * ddiv(1.0, q2));
      }
      vjp_ingrid_ff<STAGE>(g, Xs, Qs, dpx, dpq, ps.t0, ps.ts0, ps.u0, ps.us0, p, cot, gx, gq, gv, st);
      return;
    }
    const double ix = ddiv(1.0, x), iq = ddiv(1.0, q2);
    Site64 X[2], Q[2];
    for (int a = 0; a < (lowx ? 2 : 1); a++) {
      int xc = a ? ps.xc1 : ps.xc0;
      double t = a ? ps.t1 : ps.t0, s = a ? 1.0 - ps.t1 : ps.ts0;
      double dpos = (a == 0 && !lowx) ? g.xcell[4 * xc + 1] * ix : 0.0;
      make_site(X[a], g.xW + 16 * xc, t, s, xc, xc - 1, dpos);
    }
    for (int b = 0; b < (realq ? 1 : 2); b++) {
      int qc = b ? ps.qc1 : ps.qc0;
      double u = b ? ps.u1 : ps.u0, s = b ? 1.0 - ps.u1 : ps.us0;
      int row = g.qc_row[qc];
      double dpos = (b == 0 && realq) ? g.qcell[4 * row + 1] * iq : 0.0;
      make_site(Q[b], g.qW + 16 * qc, u, s, qc, row - 1, dpos);
    }
    if (cls == C_IN && g.ff) {
      vjp_ingrid_ff<STAGE>(g, X[0], Q[0], ff_of(X[0].dpos), ff_of(Q[0].dpos), ps.t0, ps.ts0, ps.u0, ps.us0, p, cot,
                           gx, gq, gv, st);
      return;
    }
    const int nsx = lowx ? 2 : 1;
    const int nsq = realq ? 1 : 2;
    const double dpx = lowx ? g.idx0 * ix : 0.0;
    // the q rule's parameter per unit Q^2: p_q = -(ln Q^2 - ln Q2max) idq_top, or rho = Q^2 / Q2min
    const double dpq = lowq ? g.inv_q2min : -g.idq_top * iq;
    double irho = 0.0, iL = 0.0;
    if (lowq) {
      irho = ddiv(1.0, ps.pq);
      iL = g.iln101;
    }
    // sites on a knot (weights (1, 0, 0, 0)): the x rule's x sites, the Q rule's Q sites but the
    // low-Q^2 rule's second one
    // the rules' point constants in float pairs (float-float-safe grids)
    const FFTabs FT{g.fflog, g.ffexp};
    RuleFF cq, cx;
    if (g.ff) {
      if (!realq) cq = rule_ff_consts(ps.pq, lowq, ps.pq, ps.lr, irho, iL);
      if (lowx) cx = rule_ff_consts(ps.px, false, 0.0, 0.0, 0.0, 0.0);
    }
    bool xk[2], qk[2];
    for (int a = 0; a < nsx; a++) xk[a] = X[a].B[1] == 0.0 && X[a].B[2] == 0.0 && X[a].B[3] == 0.0;
    for (int b = 0; b < nsq; b++) qk[b] = Q[b].B[1] == 0.0 && Q[b].B[2] == 0.0 && Q[b].B[3] == 0.0;
    // the sorted kernel's warps of points that take both rules: when all 32
    // lanes have the same class and sites (hence the same knots), each knot
    // term is summed over the warp and added by one lane (k0 + 1 of each
    // site in 14 bits)
    double *const gvc = STAGE && st ? st->gvc : gv;
    bool wsum = false;
    if (STAGE && gv && lowx && !realq && g.nx < 16383 && g.nrows < 16383) {
      const unsigned long long key =
          (unsigned long long)cls | (unsigned long long)(X[0].k0 + 1) << 4 |
          (unsigned long long)(lowx ? X[1].k0 + 1 : 0) << 18 | (unsigned long long)(Q[0].k0 + 1) << 32 |
          (unsigned long long)(realq ? 0 : Q[1].k0 + 1) << 46;
      int same = 0;
      if (__activemask() == 0xffffffffu) __match_all_sync(0xffffffffu, key, &same);
      wsum = same != 0;
    }
    double sx = 0.0, sq = 0.0;
    for (int f = 0; f < g.nf; f++) {
      const double c = cot[p * g.nf + f];
      double F[2][2], Ft[2][2], Fu[2][2];
      for (int a = 0; a < nsx; a++)
        for (int b = 0; b < nsq; b++) {
          const double *blk = g.coef + (((size_t)Q[b].c * g.nx + X[a].c) * g.nf + f) * 16;
          // x sites of the x rule are fixed (no F_t), Q sites of the Q rule too (no F_u)
          patch_site(blk, X[a], Q[b], xk[a], qk[b], !lowx, realq, F[a][b], Ft[a][b], Fu[a][b]);
        }
      // the q rule on each x site (lam_q: dA/dF(a, 0), dA/dF(a, 1), dA/dpar), then the x rule
      double A[2], l0[2], l1[2], lpar[2];
      for (int a = 0; a < nsx; a++) {
        if (!realq) {
          const RuleD R = g.ff ? rule_d_ff(F[a][0], F[a][1], cq, FT, LT, ET)
                               : rule_d(F[a][0], F[a][1], ps.pq, lowq, ps.pq, ps.lr, irho, iL, LT, ET);
          A[a] = R.v; l0[a] = R.d0; l1[a] = R.d1; lpar[a] = R.dpar;
        } else {
          A[a] = F[a][0]; l0[a] = 1.0; l1[a] = 0.0; lpar[a] = 0.0;
        }
      }
      double o0 = 1.0, o1 = 0.0, dvpx = 0.0;
      if (lowx) {
        const RuleD R = g.ff ? rule_d_ff(A[0], A[1], cx, FT, LT, ET)
                             : rule_d(A[0], A[1], ps.px, false, 0.0, 0.0, 0.0, 0.0, LT, ET);
        o0 = R.d0; o1 = R.d1; dvpx = R.dpar;
      }
      double lam[2][2];
      lam[0][0] = o0 * l0[0];
      double dx = 0.0, dq = 0.0;
      if (lowx) {
        lam[1][0] = o1 * l0[1];
        dx = dvpx * dpx;
      }
      if (!realq) {
        lam[0][1] = o0 * l1[0];
        double dpar = o0 * lpar[0];
        if (lowx) {
          lam[1][1] = o1 * l1[1];
          dpar = fma(o1, lpar[1], dpar);
        }
        dq = dpar * dpq;
      }
      for (int a = 0; a < nsx; a++)
        for (int b = 0; b < nsq; b++) {
          dx = fma(lam[a][b] * Ft[a][b], X[a].dpos, dx);
          dq = fma(lam[a][b] * Fu[a][b], Q[b].dpos, dq);
          if (STAGE && wsum) {
            // the same knots in every lane: a term that is zero in every lane is skipped
            const double m = c * lam[a][b];
            for (int bb = 0; bb < 4; bb++) {
              const int row = Q[b].k0 + bb;
              const double wq = Q[b].w[bb];
              if (!__any_sync(0xffffffffu, (__double_as_longlong(m * wq) << 1) != 0) || row < 0 || row >= g.nrows)
                continue;
              const double mq = m * wq;
              for (int aa = 0; aa < 4; aa++) {
                const int col = X[a].k0 + aa;
                const double wx = X[a].w[aa];
                if (!__any_sync(0xffffffffu, (__double_as_longlong(wx) << 1) != 0) || col < 0 || col >= g.nx)
                  continue;
                double v = mq * wx;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                if ((threadIdx.x & 31) == 0 && (__double_as_longlong(v) << 1) != 0)
                  atomicAdd(gvc + ((size_t)row * g.nx + col) * g.nf + f, v);
              }
            }
          } else if (gv) {
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
                atomicAdd(gvc + ((size_t)row * g.nx + col) * g.nf + f, mq * wx);
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
// queued per warp in three queues -- x rule only, Q rule only, both -- and
// processed 32 of one kind at a time: a warp of in-grid points never runs
// the continuation code for a few lanes, and a continuation warp runs one
// kind of rule sequence (the FP64 pipe pays for every lane of an
// instruction, so mixed kinds would run each sequence for a few lanes).
// What is left in the queues at the end goes in mixed warps of 32.
constexpr int kAdjWarps = kAdjThreads / 32;
constexpr int kAdjQ = 64;  // queue capacity: below 32 before a tile adds at most 32

__global__ void __launch_bounds__(kAdjThreads, 1)
k_vjp(GridView g, const double *__restrict__ xa, const double *__restrict__ qa, const double *__restrict__ cot,
      long long n, double *__restrict__ gx, double *__restrict__ gq, double *__restrict__ gv) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ long long queue[kAdjWarps][3][kAdjQ];
  long long *xkeys = reinterpret_cast<long long *>(smem);
  long long *qkeys = reinterpret_cast<long long *>(smem + keys_bytes(g.nx, 8));
  size_t off = keys_bytes(g.nx, 8) + keys_bytes(g.nrows, 8);
  double2 *LTt = reinterpret_cast<double2 *>(smem + off);  // the logarithm's and exponential's tables
  off += sizeof(double2) * kLogTab;
  double *LTh = reinterpret_cast<double *>(smem + off);
  off += sizeof(double) * kLogTab;
  double *ET = reinterpret_cast<double *>(smem + off);
  load_keys<double>(g, xkeys, 0);
  load_keys<double>(g, qkeys, 1);
  for (int i = threadIdx.x; i < kLogTab; i += kAdjThreads) { LTt[i] = g.tlogtab[i]; LTh[i] = g.tloghtab[i]; }
  for (int i = threadIdx.x; i < kExpTab; i += kAdjThreads) ET[i] = g.texptab[i];
  const LogTabs LT{LTt, LTh};
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  const long long kxlast = __double_as_longlong(g.xlast), kx0 = __double_as_longlong(g.x0);
  const long long kqmin = __double_as_longlong(g.q2min), kqmax = __double_as_longlong(g.q2max);
  int n0 = 0, n1 = 0, n2 = 0;  // queued points per kind (warp-uniform)
  const long long ntiles = (n + 31) / 32, nwarps = (long long)gridDim.x * kAdjWarps;
  long long tile = (long long)blockIdx.x * kAdjWarps + warp;
  // one call site: each round either drains 32 queued points of one kind, or
  // takes the in-grid points of the next tile (queueing its continuation
  // points), or drains what is left of a queue at the end (every branch is
  // warp-uniform)
  while (true) {
    long long pp = -1;
    const int full = n0 >= 32 ? 0 : n1 >= 32 ? 1 : n2 >= 32 ? 2 : -1;
    if (full >= 0) {
      const int c = (full == 0 ? n0 : full == 1 ? n1 : n2) - 32;
      pp = queue[warp][full][c + lane];
      if (full == 0) n0 = c; else if (full == 1) n1 = c; else n2 = c;
    } else if (tile < ntiles) {
      const long long p = tile * 32 + lane;
      int kind = -1;
      if (p < n) {
        const long long kx = __double_as_longlong(xa[p]), kq = __double_as_longlong(qa[p]);
        const bool valid = kq > 0 && kq < 0x7FF0000000000000LL && kx > 0 && kx <= kxlast;
        const bool fx = kx < kx0, fq = kq < kqmin || kq > kqmax;
        if (valid && (fx || fq)) kind = fx ? (fq ? 2 : 0) : 1;
        else pp = p;
      }
      const unsigned m0 = __ballot_sync(0xffffffffu, kind == 0), m1 = __ballot_sync(0xffffffffu, kind == 1),
                     m2 = __ballot_sync(0xffffffffu, kind == 2);
      if (kind == 0) queue[warp][0][n0 + __popc(m0 & lt)] = p;
      if (kind == 1) queue[warp][1][n1 + __popc(m1 & lt)] = p;
      if (kind == 2) queue[warp][2][n2 + __popc(m2 & lt)] = p;
      n0 += __popc(m0); n1 += __popc(m1); n2 += __popc(m2);
      tile += nwarps;
    } else if (n0 + n1 + n2 > 0) {  // the rest, kinds mixed, up to 32 at a time
      const int t0 = min(n0, 32), t1 = min(n1, 32 - t0), t2 = min(n2, 32 - t0 - t1);
      if (lane < t0) pp = queue[warp][0][n0 - t0 + lane];
      else if (lane < t0 + t1) pp = queue[warp][1][n1 - t1 + lane - t0];
      else if (lane < t0 + t1 + t2) pp = queue[warp][2][n2 - t2 + lane - t0 - t1];
      n0 -= t0; n1 -= t1; n2 -= t2;
    } else {
      break;
    }
    __syncwarp();
    if (pp >= 0) vjp_point<false>(g, xkeys, qkeys, LT, ET, pp, xa, qa, cot, gx, gq, gv, nullptr);
    __syncwarp();
  }
}

// ---- large batches: points sorted by cell ------------------------------------
// A counting sort puts the continuation points first, by kind (below), then
// the invalid points, then the in-grid points cell by cell.  A warp then
// takes 32 consecutive sorted points: continuation warps are of one kind (as
// with the queues above), and in-grid warps hold runs of points that share a
// cell, hence the same 16 knots.  Their knot-value gradient is contracted over the run in
// float-float on the FMA pipe,
//   dL/df_(ab, f) += sum_p c_pf w_b(u_p) w_a(t_p),
// and added with one FP64 atomic per knot and flavour per run instead of one
// per point (the per-point products were a third of an in-grid point's FP64
// work, and their atomics a stream of L2 reductions).
//
// Continuation bins: the x rule alone (bin 0), a Q rule alone (bin 1), both
// rules below (bin 2) and above the Q^2 range (bin 3).  Points that take both
// rules all add to the same few knots (x0, x1 in the bottom or top rows), so
// a warp of them sums each knot term before one atomic (without that, every
// such point's atomics went to the same addresses, one after another: 20 to
// 44 ms per 1e6 of them, against 5 to 8 ms).  The other continuation points
// spread their atomics over the rows or columns of their cells; summing
// theirs in the warp (sorted by cell) costs more FP64 additions than the
// waits it saves.
constexpr int kSortCont = 4;  // continuation bins; the invalid bin follows, then the cells
constexpr int kSortMaxBins = 65540;  // above this the grid has too many cells for runs to form
constexpr long long kSortMinN = 2048;
constexpr int kSortThreads = 128;    // three blocks per SM: 12 warps at <= 168 registers
constexpr int kStPad = 17;           // float2 per staged weight row (16 used): 2-way bank conflicts at most
constexpr int kStPadC = 18;          // float2 per staged cotangent row: 8 flavour pairs {hi, hi, lo, lo}, 16-byte rows
constexpr int kAdjCopies = 16;       // private knot-gradient copies for continuation points (at most)
constexpr size_t kAdjCopyBytes = 64u << 20;

// Sort key of a point: its continuation bin, the invalid bin, or for an
// in-grid point (bins after those) its cell, (Q cell) nx + (x cell), from
// integer range tests and searches on the raw bit patterns (no logarithm);
// counts per key in cnt.
__global__ void __launch_bounds__(256) k_adj_key(GridView g, const double *__restrict__ xa,
                                                 const double *__restrict__ qa, long long n, unsigned nb,
                                                 unsigned *__restrict__ keys, unsigned *__restrict__ cnt) {
  extern __shared__ __align__(16) unsigned char smem[];
  long long *xkeys = reinterpret_cast<long long *>(smem);
  long long *qkeys = reinterpret_cast<long long *>(smem + keys_bytes(g.nx, 8));
  load_keys<double>(g, xkeys, 0);
  load_keys<double>(g, qkeys, 1);
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const long long kxlast = __double_as_longlong(g.xlast), kx0 = __double_as_longlong(g.x0);
  const long long kqmin = __double_as_longlong(g.q2min), kqmax = __double_as_longlong(g.q2max);
  const unsigned cont = (unsigned)kSortCont;  // the invalid bin; in-grid bins follow
  // whole warps iterate together (blockDim is a multiple of 32) for the match
  for (long long base = (long long)blockIdx.x * blockDim.x; base < n; base += (long long)gridDim.x * blockDim.x) {
    const long long p = base + threadIdx.x;
    unsigned key = 0xFFFFFFFFu;
    if (p < n) {
      const long long kx = __double_as_longlong(xa[p]), kq = __double_as_longlong(qa[p]);
      const bool valid = kq > 0 && kq < 0x7FF0000000000000LL && kx > 0 && kx <= kxlast;
      const bool fx = kx < kx0, fq = kq < kqmin || kq > kqmax;
      if (!valid) {
        key = cont;
      } else if (fx || fq) {
        key = fx ? (fq ? (kq > kqmax ? 3u : 2u) : 0u) : 1u;
      } else {
        const int i = search_cell(xkeys, g.nx, g.xstep, kx);
        const int j = search_cell(qkeys, g.nrows, g.qstep, kq);
        key = cont + 1u + (unsigned)max(g.row_qc[j], 0) * (unsigned)g.nx + (unsigned)i;
      }
      key = min(key, nb - 1u);
      keys[p] = key;
    }
    const unsigned peers = __match_any_sync(0xffffffffu, key);
    if (key != 0xFFFFFFFFu && lane == __ffs(peers) - 1) atomicAdd(cnt + key, (unsigned)__popc(peers));
  }
}

// Exclusive prefix sum of cnt[0, nb) in place (one block of 1024 threads).
__global__ void __launch_bounds__(1024) k_adj_scan(unsigned *cnt, int nb) {
  __shared__ unsigned part[1024];
  const int per = (nb + 1023) / 1024;
  const int a = min((int)threadIdx.x * per, nb), b = min(a + per, nb);
  unsigned sum = 0;
  for (int i = a; i < b; i++) sum += cnt[i];
  part[threadIdx.x] = sum;
  __syncthreads();
  for (int d = 1; d < 1024; d <<= 1) {
    const unsigned v = threadIdx.x >= (unsigned)d ? part[threadIdx.x - d] : 0u;
    __syncthreads();
    part[threadIdx.x] += v;
    __syncthreads();
  }
  unsigned run = threadIdx.x ? part[threadIdx.x - 1] : 0u;
  for (int i = a; i < b; i++) {
    const unsigned c = cnt[i];
    cnt[i] = run;
    run += c;
  }
}

// perm[cursor[key]++] = p, one atomic per key per warp.
__global__ void __launch_bounds__(256) k_adj_place(const unsigned *__restrict__ keys, long long n,
                                                   unsigned *__restrict__ cursor, unsigned *__restrict__ perm) {
  const int lane = threadIdx.x & 31;
  for (long long base = (long long)blockIdx.x * blockDim.x; base < n; base += (long long)gridDim.x * blockDim.x) {
    const long long p = base + threadIdx.x;
    const unsigned key = p < n ? keys[p] : 0xFFFFFFFFu;
    const unsigned peers = __match_any_sync(0xffffffffu, key);
    const int leader = __ffs(peers) - 1;
    unsigned at = 0;
    if (key != 0xFFFFFFFFu && lane == leader) at = atomicAdd(cursor + key, (unsigned)__popc(peers));
    at = __shfl_sync(0xffffffffu, at, leader);
    if (key != 0xFFFFFFFFu) perm[at + __popc(peers & ((1u << lane) - 1u))] = (unsigned)p;
  }
}

// One warp per 32 sorted points, tiles handed out in sorted order by a
// counter (the costly continuation tiles first, the cheap in-grid ones fill
// in at the end).  With GV, each run of lanes sharing a cell contracts its
// staged terms: lane l owns knot m = l mod 16 of the cell and flavours
// l / 16, l / 16 + 2, ... (at most 16 flavours).  Blocks of four warps,
// three per SM: 12 warps at <= 168 registers hide more of the FP64 latency
// than 8 at 254 (1.66 -> 1.56 ms per 1e6 points; 16 warps at 128 registers,
// with more spills, measured the same as 12).
template <bool GV>
__global__ void __launch_bounds__(kSortThreads, 3)
k_vjp_sorted(GridView g, const double *__restrict__ xa, const double *__restrict__ qa,
             const double *__restrict__ cot, long long n, const unsigned *__restrict__ perm,
             unsigned long long *__restrict__ next_tile, double *__restrict__ gx, double *__restrict__ gq,
             double *__restrict__ gv, double *__restrict__ gvp, int ncopy, long long pstride) {
  extern __shared__ __align__(16) unsigned char smem[];
  long long *xkeys = reinterpret_cast<long long *>(smem);
  long long *qkeys = reinterpret_cast<long long *>(smem + keys_bytes(g.nx, 8));
  size_t off = keys_bytes(g.nx, 8) + keys_bytes(g.nrows, 8);
  double2 *LTt = reinterpret_cast<double2 *>(smem + off);
  off += sizeof(double2) * kLogTab;
  double *LTh = reinterpret_cast<double *>(smem + off);
  off += sizeof(double) * kLogTab;
  double *ET = reinterpret_cast<double *>(smem + off);
  off += sizeof(double) * kExpTab;
  off = (off + 15) & ~(size_t)15;
  float2 *stw = reinterpret_cast<float2 *>(smem + off);  // [warp][lane][kStPad] weights
  float2 *stc = stw + kSortThreads * kStPad;              // [warp][lane][kStPadC] cotangent pairs
  load_keys<double>(g, xkeys, 0);
  load_keys<double>(g, qkeys, 1);
  for (int i = threadIdx.x; i < kLogTab; i += kSortThreads) { LTt[i] = g.tlogtab[i]; LTh[i] = g.tloghtab[i]; }
  for (int i = threadIdx.x; i < kExpTab; i += kSortThreads) ET[i] = g.texptab[i];
  const LogTabs LT{LTt, LTh};
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float2 *wrow = stw + (size_t)threadIdx.x * kStPad, *crow = stc + (size_t)threadIdx.x * kStPadC;
  const float2 *wwarp = stw + (size_t)warp * 32 * kStPad, *cwarp = stc + (size_t)warp * 32 * kStPadC;
  const long long ntiles = (n + 31) / 32;
  while (true) {
    unsigned long long t = 0;
    if (lane == 0) t = atomicAdd(next_tile, 1ull);
    const long long tile = (long long)__shfl_sync(0xffffffffu, t, 0);
    if (tile >= ntiles) break;
    const long long pos = tile * 32 + lane;
    Staged st{wrow, crow, -1, 0, 0, false, ncopy > 0 ? gvp + (tile % ncopy) * pstride : gv};
    if (pos < n) vjp_point<true>(g, xkeys, qkeys, LT, ET, (long long)perm[pos], xa, qa, cot, gx, gq, gv, &st);
    if (GV) {
      __syncwarp();
      // lane: knot m, flavours 8 fh .. 8 fh + 7 as four pairs, each pair's
      // sum in one packed (f32x2) float-float chain -- the steps of ff_acc
      // per half
      const int m = lane & 15, fh = lane >> 4;
      unsigned todo = __ballot_sync(0xffffffffu, st.ing);
      while (todo) {  // one run of lanes sharing a cell at a time
        const int leader = __ffs(todo) - 1;
        const int cell = __shfl_sync(0xffffffffu, st.cell, leader);
        const int xk0 = __shfl_sync(0xffffffffu, st.xk0, leader);
        const int qk0 = __shfl_sync(0xffffffffu, st.qk0, leader);
        const unsigned run = __ballot_sync(0xffffffffu, st.ing && st.cell == cell);
        todo &= ~run;
        float2 sh[4], sl[4];
#pragma unroll
        for (int k = 0; k < 4; k++) sh[k] = sl[k] = make_float2(0.f, 0.f);
        for (unsigned r = run; r; r &= r - 1) {
          const int q = __ffs(r) - 1;
          const float2 w = wwarp[q * kStPad + m];
          const float2 wh = make_float2(w.x, w.x), wl = make_float2(w.y, w.y);
          const float4 *cq = reinterpret_cast<const float4 *>(cwarp + q * kStPadC) + 4 * fh;
#pragma unroll
          for (int k = 0; k < 4; k++) {
            const float4 cc = cq[k];
            const float2 ch = make_float2(cc.x, cc.y), cl = make_float2(cc.z, cc.w);
            const float2 ph = __fmul2_rn(wh, ch);
            float2 pe = __ffma2_rn(wh, ch, neg2(ph));
            pe = __ffma2_rn(wh, cl, __ffma2_rn(wl, ch, pe));
            const float2 t = __fadd2_rn(sh[k], ph);
            const float2 bp = __fadd2_rn(t, neg2(sh[k]));
            const float2 err = __fadd2_rn(__fadd2_rn(sh[k], neg2(__fadd2_rn(t, neg2(bp)))), __fadd2_rn(ph, neg2(bp)));
            sh[k] = t;
            sl[k] = __fadd2_rn(sl[k], __fadd2_rn(err, pe));
          }
        }
        const int row = qk0 + (m >> 2), col = xk0 + (m & 3);
        if (row >= 0 && row < g.nrows && col >= 0 && col < g.nx) {
          double *dst = gv + ((size_t)row * g.nx + col) * g.nf;
#pragma unroll
          for (int k = 0; k < 4; k++) {
            const int f = 8 * fh + 2 * k;
            if (f < g.nf) atomicAdd(dst + f, f2d(sh[k].x) + f2d(sl[k].x));
            if (f + 1 < g.nf) atomicAdd(dst + f + 1, f2d(sh[k].y) + f2d(sl[k].y));
          }
        }
      }
      __syncwarp();
    }
  }
}

// gv[i] += sum over the private copies of their element i (copies zeroed
// before the sorted kernel; continuation points' knot terms went there).
__global__ void __launch_bounds__(256) k_adj_fold(double *__restrict__ gv, const double *__restrict__ gvp,
                                                  int ncopy, long long pstride) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < pstride;
       i += (long long)gridDim.x * blockDim.x) {
    double sum = 0.0;
    for (int k = 0; k < ncopy; k++) sum += gvp[k * pstride + i];
    if ((__double_as_longlong(sum) << 1) != 0) gv[i] += sum;
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
  if (sms < 1) sms = 1;
  const size_t kbytes = keys_bytes(g.nx, 8) + keys_bytes(g.nrows, 8);
  const size_t smem = kbytes + (sizeof(double2) + sizeof(double)) * kLogTab + sizeof(double) * kExpTab;
  const long long nb = kSortCont + 1 + (long long)(g.nqc + 1) * g.nx;

  // large batches on a float-float-safe grid: sorted by cell (see k_vjp_sorted)
  if ((long long)n >= kSortMinN && n < (1ull << 31) && g.ff && g.nf <= 16 && nb <= kSortMaxBins) {
    static LaunchCache cache_t, cache_f;
    const size_t ssmem = ((smem + 15) & ~(size_t)15) + sizeof(float2) * kSortThreads * (kStPad + kStPadC);
    LaunchCache &cache = grad_values ? cache_t : cache_f;
    const int per_sm = grad_values ? cache.blocks_per_sm(k_vjp_sorted<true>, kSortThreads, ssmem, false)
                                   : cache.blocks_per_sm(k_vjp_sorted<false>, kSortThreads, ssmem, false);
    void *buf = nullptr;
    const size_t cnt_bytes = ((size_t)nb * sizeof(unsigned) + 15) / 16 * 16;
    const size_t sort_bytes = cnt_bytes + 16 + 2 * ((n * sizeof(unsigned) + 15) / 16 * 16);
    // private copies of the knot gradient for the continuation points' atomics
    // (they add to the few knots next to the grid's edges, and spreading them
    // over copies spreads the queues on those addresses)
    const long long pstride = (long long)g.nrows * g.nx * g.nf;
    int ncopy = 0;
    if (grad_values && pstride > 0) {
      ncopy = kAdjCopies;
      while (ncopy > 1 && ((size_t)ncopy * pstride * sizeof(double) > kAdjCopyBytes ||
                           sort_bytes + (size_t)ncopy * pstride * sizeof(double) > scratch_limit()))
        ncopy >>= 1;
      if (ncopy < 2) ncopy = 0;
    }
    const size_t copy_bytes = (size_t)ncopy * pstride * sizeof(double);
    const size_t bytes = sort_bytes + copy_bytes;
    cudaMemPool_t pool = bytes <= scratch_limit() ? sort_pool(dev) : nullptr;
    if (per_sm >= 1 && pool && cudaMallocFromPoolAsync(&buf, bytes, pool, stream) == cudaSuccess) {
      unsigned *cnt = static_cast<unsigned *>(buf);
      auto *next_tile = reinterpret_cast<unsigned long long *>(static_cast<char *>(buf) + cnt_bytes);
      double *gvp = reinterpret_cast<double *>(static_cast<char *>(buf) + cnt_bytes + 16);
      unsigned *keys = reinterpret_cast<unsigned *>(static_cast<char *>(buf) + cnt_bytes + 16 + copy_bytes);
      unsigned *perm = keys + (n * sizeof(unsigned) + 15) / 16 * 4;
      int rc = PDF_OK;
      if (cudaMemsetAsync(buf, 0, cnt_bytes + 16 + copy_bytes, stream) != cudaSuccess)
        rc = set_error(PDF_ERR_CUDA, "xfxq2_all_flavours_vjp: scratch");
      const unsigned sblocks = (unsigned)std::min<long long>(((long long)n + 255) / 256, 8LL * sms);
      if (!rc) {
        k_adj_key<<<sblocks, 256, kbytes, stream>>>(g, x, q2, (long long)n, (unsigned)nb, keys, cnt);
        k_adj_scan<<<1, 1024, 0, stream>>>(cnt, (int)nb);
        k_adj_place<<<sblocks, 256, 0, stream>>>(keys, (long long)n, cnt, perm);
        const unsigned blocks =
            (unsigned)std::min<long long>(((long long)n + kSortThreads - 1) / kSortThreads, (long long)sms * per_sm);
        if (grad_values) {
          k_vjp_sorted<true><<<blocks, kSortThreads, ssmem, stream>>>(g, x, q2, cot, (long long)n, perm, next_tile,
                                                                      grad_x, grad_q2, grad_values, gvp, ncopy,
                                                                      pstride);
          if (ncopy > 0)
            k_adj_fold<<<(unsigned)std::min<long long>((pstride + 255) / 256, 4LL * sms), 256, 0, stream>>>(
                grad_values, gvp, ncopy, pstride);
        } else {
          k_vjp_sorted<false><<<blocks, kSortThreads, ssmem, stream>>>(g, x, q2, cot, (long long)n, perm, next_tile,
                                                                       grad_x, grad_q2, grad_values, nullptr, 0, 0);
        }
        rc = check_launch("xfxq2_all_flavours_vjp sorted kernels");
      }
      cudaFreeAsync(buf, stream);
      return rc;
    }
    cudaGetLastError();  // no scratch: the unsorted kernel below needs none
  }

  // one resident block per SM (its registers fill the SM), each warp taking many
  // tiles so that its continuation queues fill to whole warps
  long long blocks = ((long long)n + kAdjThreads - 1) / kAdjThreads;
  if (blocks > sms) blocks = sms;
  k_vjp<<<(unsigned)blocks, kAdjThreads, smem, stream>>>(g, x, q2, cot, (long long)n, grad_x, grad_q2,
                                                         grad_values);
  return check_launch("xfxq2_all_flavours_vjp kernel");
}
