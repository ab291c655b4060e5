/*
 * pdf_oracle.c -- plain, slow FP64 CPU oracle for the PDFFlow hot path.
 *
 * TEST INFRASTRUCTURE.  Only the tests, the smoke check and the CPU-baseline
 * leg of the benchmark may load this file's library.  It shares no code,
 * header, table or constant with the CUDA path.
 *
 * What it computes (PDFFlow, Sec. 2.2 and 2.3):
 *   - x f(x, Q^2) by log-bicubic interpolation of tabulated knot values in
 *     (ln x, ln Q^2), following the LHAPDF6 prescription the paper adopts
 *     (Sec. 2.2): cubic Hermite segments whose knot tangents are finite
 *     differences of the knot values, x direction first at each needed Q
 *     row, then the Q direction on the interpolated rows;
 *   - Q subgrids split at flavour thresholds are interpolated independently
 *     and no difference stencil crosses a subgrid boundary (Sec. 2.2,
 *     "special care ... close to quark mass thresholds and grid x edges");
 *   - extrapolation outside the grid (the EXTRAPOLATE box of Fig. 1; the
 *     paper prints no rule, the continuation rules below are the reading);
 *   - alpha_s(Q^2) by log-cubic interpolation of the (Q, alpha_s) nodes with
 *     constant extrapolation, subgrids split at repeated nodes (Sec. 2.3).
 *
 * Readings where the paper is silent (each one is listed in the design notes):
 *   R-coord  interpolate the stored xf values in t = ln x, ln Q^2.
 *   R-slope  knot slope = mean of the two adjacent secant slopes; one-sided
 *            secant at the first/last knot of the x grid and of each Q
 *            subgrid; Hermite tangent = slope * cell width.
 *   R-order  x first, then Q.
 *   R-ends   the position inside a cell is carried as the pair (t, 1 - t),
 *            each taken from its own knot, t = (ln x - ln x_i)/d and
 *            1 - t = (ln x_{i+1} - ln x)/d, and the Hermite basis is
 *            evaluated in factored form; so a point within rounding of the
 *            far knot (x -> 1, where xf ~ (1 - t)) keeps its relative
 *            precision.  The cubic is the textbook one.
 *   R-ties   cells are chosen on the raw inputs (x, Q^2) against the raw
 *            knots: a point on an interior knot belongs to the cell on its
 *            right; the last knot closes the last cell; Q^2 on a subgrid
 *            boundary belongs to the upper subgrid.
 *   R-extra  low x: G0, G1 = values at the two lowest x knots;
 *              p = (ln x - ln x0)/(ln x1 - ln x0);
 *              xf = G0 (G1/G0)^p if G0 > 0 and G1 > 0, else G0 + (G1-G0) p.
 *            high Q^2: the same pair rule in ln Q^2 from the last knot and the
 *              one below it.
 *            low Q^2: f0 = F(x, Q2min), f1 = F(x, 1.01 Q2min),
 *              gamma = ln(f1/f0)/ln(1.01) if both > 0, else 1;
 *              rho = Q^2/Q2min; xf = f0 rho^(gamma rho + 1 - rho).
 *            corners: the Q rule at x0 and x1, then the low-x rule.
 *            invalid (x <= 0, x > last x knot, Q^2 <= 0, Q^2 = inf, NaN): NaN.
 *   R-alphas alpha_s nodes interpolated in ln Q^2 with the R-slope stencil
 *            inside each subgrid; constant below the first and above the last
 *            node; a Q^2 equal to a repeated node belongs to the upper subgrid.
 *
 * Every value is carried as a quadruple (v, d, m, s):
 *   v  the FP64 value;
 *   d  its forward-mode derivative with respect to one seeded input (x, Q^2
 *      or one knot value) -- the gradient oracle;
 *   m  a running first-order rounding-error bound in units of the unit
 *      roundoff (|computed - exact| <~ m * 2^-53), used to flag branch
 *      decisions that rounding could flip;
 *   s  the data mass: first-order propagation of the data's absolute size
 *      through the same expression (a datum gives |f|; a + b and a - b give
 *      s_a + s_b; a b gives |b| s_a + |a| s_b; a / b gives
 *      (s_a + |a/b| s_b) / |b|; ln a gives s_a / |a|; e^a gives e^a s_a).
 *      For an in-grid point it is sum_ab P_ab |f_ab|, P_ab the sum of the
 *      magnitudes of the coefficients along every path from knot (a, b) to
 *      the result, so s >= sum_ab |W_ab f_ab| >= |xf| with W_ab = d xf/d f_ab;
 *      on a grid of constant value C, s = |C| R(t) R(u) with
 *      R(t) = 1 + a0 t (1-t)^2 + a1 t^2 (1-t), a0 = 1 + d_i / d_(i-1) and
 *      a1 = 1 + d_i / d_(i+1) for cell widths d (2 where the tangent is a
 *      one-sided secant).  Through a log-linear continuation from knot
 *      values it grows to |xf| (1 + 2|p|).
 *      It is the scale of a relative error near zero crossings of xf, where
 *      |xf| itself is no scale, and the size of the rounding any evaluation
 *      order of the same formula can make.
 *
 * Build: gcc -O2 -fopenmp -ffp-contract=off -shared -fPIC (no FMA
 * contraction, so x86-64 and aarch64 hosts give identical bits).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------ */
/* value / derivative / error-mass arithmetic                          */
/* ------------------------------------------------------------------ */

typedef struct { double v, d, m, s; } num;

static num cst(double c) { num r = {c, 0.0, 0.0, 0.0}; return r; }       /* exact constant  */
static num dat(double c) { num r = {c, 0.0, 0.0, fabs(c)}; return r; }   /* tabulated datum */
static num add(num a, num b) {
  num r; r.v = a.v + b.v; r.d = a.d + b.d; r.m = a.m + b.m + fabs(r.v); r.s = a.s + b.s; return r;
}
static num sub(num a, num b) {
  num r; r.v = a.v - b.v; r.d = a.d - b.d; r.m = a.m + b.m + fabs(r.v); r.s = a.s + b.s; return r;
}
static num mul(num a, num b) {
  num r; r.v = a.v * b.v; r.d = a.d * b.v + a.v * b.d;
  r.m = fabs(b.v) * a.m + fabs(a.v) * b.m + fabs(r.v);
  r.s = fabs(b.v) * a.s + fabs(a.v) * b.s; return r;
}
static num dvd(num a, num b) {
  num r; r.v = a.v / b.v; r.d = (a.d - r.v * b.d) / b.v;
  r.m = (a.m + fabs(r.v) * b.m) / fabs(b.v) + fabs(r.v);
  r.s = (a.s + fabs(r.v) * b.s) / fabs(b.v); return r;
}
static num nlog(num a) {
  num r; r.v = log(a.v); r.d = a.d / a.v; r.m = a.m / fabs(a.v) + fabs(r.v); r.s = a.s / fabs(a.v); return r;
}
static num nexp(num a) {
  num r; r.v = exp(a.v); r.d = r.v * a.d; r.m = fabs(r.v) * (a.m + 1.0); r.s = fabs(r.v) * a.s; return r;
}
static num nan_num(void) { num r = {NAN, NAN, NAN, NAN}; return r; }

/* ------------------------------------------------------------------ */
/* prepared grid                                                        */
/* ------------------------------------------------------------------ */

typedef struct og {
  int nx; double *xk; num *lx;       /* x knots and their logs              */
  int nsub; int *first; int *nq;     /* subgrid s = rows first[s] .. +nq-1  */
  int nrows; double *q2k; num *lq;   /* Q^2 knots (concatenated) and logs   */
  int nf; double *val;               /* [row][ix][f]                        */
  int na; double *aq2; double *aval; num *alq;  /* alpha_s nodes             */
} og;

/* What the forward-mode derivative is taken with respect to. */
enum { WRT_NONE = 0, WRT_X = 1, WRT_Q2 = 2, WRT_KNOT = 3 };
typedef struct {
  int wrt, row, ix;      /* WRT_KNOT: the knot (row, ix) of the column asked for */
  int *rec; int nrec;    /* optional list of (row, ix) knots read, for gradients */
  int marginal;          /* set when a positivity test is within rounding of 0   */
} ctx;

static num knot(const og *g, int row, int ix, int f, ctx *c) {
  num r = dat(g->val[((size_t)row * g->nx + ix) * g->nf + f]);
  r.d = (c->wrt == WRT_KNOT && c->row == row && c->ix == ix) ? 1.0 : 0.0;
  if (c->rec) {
    int seen = 0;
    for (int k = 0; k < c->nrec; k++)
      if (c->rec[2 * k] == row && c->rec[2 * k + 1] == ix) { seen = 1; break; }
    if (!seen) { c->rec[2 * c->nrec] = row; c->rec[2 * c->nrec + 1] = ix; c->nrec++; }
  }
  return r;
}

void og_free(og *g) {
  if (!g) return;
  free(g->xk); free(g->lx); free(g->first); free(g->nq); free(g->q2k); free(g->lq);
  free(g->val); free(g->aq2); free(g->aval); free(g->alq); free(g);
}

static num lognum(double k) { num r = {log(k), 0.0, 0.0, 0.0}; r.m = fabs(r.v); return r; }

/* Copy and check a grid.  *err: 0 ok, else a negative code. */
og *og_prepare(int nx, const double *xk, int nsub, const int *nq, const double *q2k,
               int nf, const double *val, int na, const double *aq2, const double *aval,
               int *err) {
  *err = 0;
  if (nx < 2 || nsub < 1 || nf < 1 || na < 0) { *err = -1; return NULL; }
  for (int i = 0; i < nx; i++) {
    if (!(xk[i] > 0.0) || !(xk[i] <= 1.0)) { *err = -2; return NULL; }
    if (i > 0 && !(xk[i] > xk[i - 1])) { *err = -2; return NULL; }
  }
  int nrows = 0;
  for (int s = 0; s < nsub; s++) {
    if (nq[s] < 2) { *err = -3; return NULL; }
    nrows += nq[s];
  }
  int r0 = 0;
  for (int s = 0; s < nsub; s++) {
    for (int j = r0; j < r0 + nq[s]; j++) {
      if (!(q2k[j] > 0.0) || !isfinite(q2k[j])) { *err = -3; return NULL; }
      if (j > r0 && !(q2k[j] > q2k[j - 1])) { *err = -3; return NULL; }
    }
    if (s > 0 && q2k[r0] != q2k[r0 - 1]) { *err = -3; return NULL; }
    r0 += nq[s];
  }
  if (!(q2k[nrows - 1] >= 1.01 * q2k[0])) { *err = -3; return NULL; }
  for (size_t k = 0; k < (size_t)nrows * nx * nf; k++)
    if (!isfinite(val[k])) { *err = -4; return NULL; }
  if (na > 0) {
    if (na < 2) { *err = -5; return NULL; }
    int run = 1;
    for (int k = 0; k < na; k++) {
      if (!(aq2[k] > 0.0) || !isfinite(aq2[k]) || !isfinite(aval[k])) { *err = -5; return NULL; }
      if (k > 0) {
        if (aq2[k] < aq2[k - 1]) { *err = -5; return NULL; }
        if (aq2[k] == aq2[k - 1]) { if (run < 2) { *err = -5; return NULL; } run = 1; }
        else run++;
      }
    }
    if (run < 2) { *err = -5; return NULL; }
  }

  og *g = (og *)calloc(1, sizeof(og));
  g->nx = nx; g->nsub = nsub; g->nrows = nrows; g->nf = nf; g->na = na;
  g->xk = malloc(sizeof(double) * nx); memcpy(g->xk, xk, sizeof(double) * nx);
  g->lx = malloc(sizeof(num) * nx);
  for (int i = 0; i < nx; i++) g->lx[i] = lognum(xk[i]);
  g->first = malloc(sizeof(int) * nsub); g->nq = malloc(sizeof(int) * nsub);
  r0 = 0;
  for (int s = 0; s < nsub; s++) { g->first[s] = r0; g->nq[s] = nq[s]; r0 += nq[s]; }
  g->q2k = malloc(sizeof(double) * nrows); memcpy(g->q2k, q2k, sizeof(double) * nrows);
  g->lq = malloc(sizeof(num) * nrows);
  for (int j = 0; j < nrows; j++) g->lq[j] = lognum(q2k[j]);
  size_t nv = (size_t)nrows * nx * nf;
  g->val = malloc(sizeof(double) * nv); memcpy(g->val, val, sizeof(double) * nv);
  if (na > 0) {
    g->aq2 = malloc(sizeof(double) * na); memcpy(g->aq2, aq2, sizeof(double) * na);
    g->aval = malloc(sizeof(double) * na); memcpy(g->aval, aval, sizeof(double) * na);
    g->alq = malloc(sizeof(num) * na);
    for (int k = 0; k < na; k++) g->alq[k] = lognum(aq2[k]);
  }
  return g;
}

/* ------------------------------------------------------------------ */
/* 1-D building blocks                                                  */
/* ------------------------------------------------------------------ */

/* Cubic Hermite segment on t in [0, 1] with end values f0, f1 and end
 * tangents m0, m1 (already multiplied by the cell width); tm = 1 - t.
 * Basis h00 = 2t^3 - 3t^2 + 1, h01 = -2t^3 + 3t^2, h10 = t^3 - 2t^2 + t,
 * h11 = t^3 - t^2, written in factored form:
 * h00 = (1 + 2t) tm^2, h01 = t^2 (1 + 2 tm), h10 = t tm^2, h11 = -t^2 tm. */
static num hermite(num t, num tm, num f0, num f1, num m0, num m1) {
  num t2 = mul(t, t), tm2 = mul(tm, tm);
  num h00 = mul(add(cst(1.0), mul(cst(2.0), t)), tm2);
  num h01 = mul(t2, add(cst(1.0), mul(cst(2.0), tm)));
  num h10 = mul(t, tm2);
  num h11 = sub(cst(0.0), mul(t2, tm));
  return add(add(mul(h00, f0), mul(h01, f1)), add(mul(h10, m0), mul(h11, m1)));
}

/* Knot slope from a 1-D sequence f[lo..hi] at knots l[lo..hi] (R-slope). */
static num secant(num fa, num fb, num la, num lb) { return dvd(sub(fb, fa), sub(lb, la)); }

/* x-direction interpolation of knot row `row` in cell i at parameter t
 * (tm = 1 - t). */
static num row_interp(const og *g, int row, int i, num t, num tm, int f, ctx *c) {
  int n = g->nx;
  num fi = knot(g, row, i, f, c), fi1 = knot(g, row, i + 1, f, c);
  num s0, s1;
  if (i == 0) s0 = secant(fi, fi1, g->lx[0], g->lx[1]);
  else s0 = mul(cst(0.5), add(secant(knot(g, row, i - 1, f, c), fi, g->lx[i - 1], g->lx[i]),
                               secant(fi, fi1, g->lx[i], g->lx[i + 1])));
  if (i + 1 == n - 1) s1 = secant(fi, fi1, g->lx[i], g->lx[i + 1]);
  else s1 = mul(cst(0.5), add(secant(fi, fi1, g->lx[i], g->lx[i + 1]),
                               secant(fi1, knot(g, row, i + 2, f, c), g->lx[i + 1], g->lx[i + 2])));
  num dx = sub(g->lx[i + 1], g->lx[i]);
  return hermite(t, tm, fi, fi1, mul(dx, s0), mul(dx, s1));
}

/* ------------------------------------------------------------------ */
/* in-grid log-bicubic interpolation F(x, Q^2)                          */
/* requires x0 <= x <= x_last and Q2min <= Q^2 <= Q2max                 */
/* ------------------------------------------------------------------ */

static num interp2(const og *g, num X, num Q2, int f, ctx *c) {
  /* cells by linear scan on the raw values (R-ties) */
  int i = 0;
  while (i + 1 < g->nx - 1 && g->xk[i + 1] <= X.v) i++;
  int s = 0;
  while (s + 1 < g->nsub && g->q2k[g->first[s + 1]] <= Q2.v) s++;
  int j0 = g->first[s], j1 = g->first[s] + g->nq[s] - 1;
  int j = j0;
  while (j + 1 < j1 && g->q2k[j + 1] <= Q2.v) j++;

  num lxv = nlog(X), lqv = nlog(Q2);
  num dx = sub(g->lx[i + 1], g->lx[i]), dq = sub(g->lq[j + 1], g->lq[j]);
  num t = dvd(sub(lxv, g->lx[i]), dx), tm = dvd(sub(g->lx[i + 1], lxv), dx);  /* R-ends */
  num u = dvd(sub(lqv, g->lq[j]), dq), um = dvd(sub(g->lq[j + 1], lqv), dq);

  /* x direction on the rows the Q stencil needs (R-order) */
  num gj = row_interp(g, j, i, t, tm, f, c);
  num gj1 = row_interp(g, j + 1, i, t, tm, f, c);
  num s0, s1;
  if (j == j0) s0 = secant(gj, gj1, g->lq[j], g->lq[j + 1]);
  else s0 = mul(cst(0.5), add(secant(row_interp(g, j - 1, i, t, tm, f, c), gj, g->lq[j - 1], g->lq[j]),
                               secant(gj, gj1, g->lq[j], g->lq[j + 1])));
  if (j + 1 == j1) s1 = secant(gj, gj1, g->lq[j], g->lq[j + 1]);
  else s1 = mul(cst(0.5), add(secant(gj, gj1, g->lq[j], g->lq[j + 1]),
                               secant(gj1, row_interp(g, j + 2, i, t, tm, f, c), g->lq[j + 1], g->lq[j + 2])));
  return hermite(u, um, gj, gj1, mul(dq, s0), mul(dq, s1));
}

/* ------------------------------------------------------------------ */
/* extrapolation (R-extra)                                              */
/* ------------------------------------------------------------------ */

#define MARGIN 256.0 * 1.1102230246251565e-16  /* 256 unit roundoffs */

static int positive(num a, ctx *c) {
  if (fabs(a.v) <= MARGIN * a.m) c->marginal = 1;
  return a.v > 0.0;
}

/* Continue from the value g0 at one knot (p = 0) using the next knot's
 * value g1 (p = 1): log-linear when both are positive, else linear. */
static num pair_rule(num g0, num g1, num p, ctx *c) {
  int pos0 = positive(g0, c), pos1 = positive(g1, c);
  if (pos0 && pos1) return mul(g0, nexp(mul(p, nlog(dvd(g1, g0)))));
  return add(g0, mul(sub(g1, g0), p));
}

/* Value at an in-range x for any Q^2: interpolation or a Q rule. */
static num q_rule(const og *g, num X, num Q2, int f, ctx *c) {
  double q2min = g->q2k[0], q2max = g->q2k[g->nrows - 1];
  if (Q2.v >= q2min && Q2.v <= q2max) return interp2(g, X, Q2, f, c);
  if (Q2.v > q2max) {
    int n = g->nrows - 1;
    num gN = interp2(g, X, cst(g->q2k[n]), f, c);
    num gM = interp2(g, X, cst(g->q2k[n - 1]), f, c);
    num p = dvd(sub(nlog(Q2), g->lq[n]), sub(g->lq[n - 1], g->lq[n]));
    return pair_rule(gN, gM, p, c);
  }
  /* low Q^2: anomalous-dimension continuation */
  num f0 = interp2(g, X, cst(q2min), f, c);
  num f1 = interp2(g, X, cst(1.01 * q2min), f, c);
  int pos0 = positive(f0, c), pos1 = positive(f1, c);
  num gam = cst(1.0);
  if (pos0 && pos1) gam = dvd(nlog(dvd(f1, f0)), lognum(1.01));
  num rho = dvd(Q2, cst(q2min));
  num ex = sub(add(mul(gam, rho), cst(1.0)), rho);
  return mul(f0, nexp(mul(ex, nlog(rho))));
}

static num xf_one(const og *g, double x, double q2, int f, ctx *c) {
  if (!(x > 0.0) || !(x <= g->xk[g->nx - 1]) || !(q2 > 0.0) || !(q2 < INFINITY)) return nan_num();
  num X = {x, c->wrt == WRT_X ? 1.0 : 0.0, 0.0, 0.0};
  num Q2 = {q2, c->wrt == WRT_Q2 ? 1.0 : 0.0, 0.0, 0.0};
  if (x >= g->xk[0]) return q_rule(g, X, Q2, f, c);
  num G0 = q_rule(g, cst(g->xk[0]), Q2, f, c);
  num G1 = q_rule(g, cst(g->xk[1]), Q2, f, c);
  num p = dvd(sub(nlog(X), g->lx[0]), sub(g->lx[1], g->lx[0]));
  return pair_rule(G0, G1, p, c);
}

/* ------------------------------------------------------------------ */
/* alpha_s (R-alphas)                                                   */
/* ------------------------------------------------------------------ */

static num alphas_one(const og *g, double q2, int wrt_q2) {
  if (g->na == 0 || !(q2 > 0.0) || !(q2 < INFINITY)) return nan_num();
  if (q2 < g->aq2[0]) return dat(g->aval[0]);
  if (q2 > g->aq2[g->na - 1]) return dat(g->aval[g->na - 1]);
  /* subgrid: the last run start a0 (index 0 or a repeated node) with aq2[a0] <= q2 */
  int a0 = 0;
  for (int k = 1; k < g->na; k++)
    if (g->aq2[k] == g->aq2[k - 1] && g->aq2[k] <= q2) a0 = k;
  int a1 = a0;
  while (a1 + 1 < g->na && g->aq2[a1 + 1] > g->aq2[a1]) a1++;
  int j = a0;
  while (j + 1 < a1 && g->aq2[j + 1] <= q2) j++;

  num Q2 = {q2, wrt_q2 ? 1.0 : 0.0, 0.0, 0.0};
  const num *l = g->alq;
  num fj = dat(g->aval[j]), fj1 = dat(g->aval[j + 1]);
  num lqv = nlog(Q2), dq = sub(l[j + 1], l[j]);
  num u = dvd(sub(lqv, l[j]), dq), um = dvd(sub(l[j + 1], lqv), dq);
  num s0, s1;
  if (j == a0) s0 = secant(fj, fj1, l[j], l[j + 1]);
  else s0 = mul(cst(0.5), add(secant(dat(g->aval[j - 1]), fj, l[j - 1], l[j]), secant(fj, fj1, l[j], l[j + 1])));
  if (j + 1 == a1) s1 = secant(fj, fj1, l[j], l[j + 1]);
  else s1 = mul(cst(0.5), add(secant(fj, fj1, l[j], l[j + 1]), secant(fj1, dat(g->aval[j + 2]), l[j + 1], l[j + 2])));
  return hermite(u, um, fj, fj1, mul(dq, s0), mul(dq, s1));
}

/* ------------------------------------------------------------------ */
/* exported batch calls                                                 */
/* ------------------------------------------------------------------ */

static int threads(int nthreads) {
#ifdef _OPENMP
  return nthreads > 0 ? nthreads : omp_get_max_threads();
#else
  (void)nthreads; return 1;
#endif
}

/* Values of columns cols[0..ncols) at n points: out_v/out_s are [n][ncols]
 * (out_s, the data mass, and out_flag may be NULL).  out_flag = 1 where a
 * positivity test of an extrapolation rule was within rounding of zero. */
void og_xfxq2(const og *g, int ncols, const int *cols, const double *x, const double *q2, long n,
              double *out_v, double *out_s, unsigned char *out_flag, int nthreads) {
#pragma omp parallel for schedule(dynamic, 64) num_threads(threads(nthreads))
  for (long p = 0; p < n; p++) {
    for (int k = 0; k < ncols; k++) {
      ctx c; memset(&c, 0, sizeof c);
      num r = xf_one(g, x[p], q2[p], cols[k], &c);
      out_v[p * ncols + k] = r.v;
      if (out_s) out_s[p * ncols + k] = r.s;
      if (out_flag) out_flag[p * ncols + k] = (unsigned char)c.marginal;
    }
  }
}

/* d xf / dx (wrt = 1) or d xf / dQ^2 (wrt = 2), [n][ncols]. */
void og_dxfxq2(const og *g, int wrt, int ncols, const int *cols, const double *x, const double *q2,
               long n, double *out_d, int nthreads) {
#pragma omp parallel for schedule(dynamic, 64) num_threads(threads(nthreads))
  for (long p = 0; p < n; p++) {
    for (int k = 0; k < ncols; k++) {
      ctx c; memset(&c, 0, sizeof c); c.wrt = wrt == 1 ? WRT_X : WRT_Q2;
      out_d[p * ncols + k] = xf_one(g, x[p], q2[p], cols[k], &c).d;
    }
  }
}

/* Knot-value gradient of L = sum_p sum_f cot[p][f] xf_f(x_p, Q2_p):
 * gvals[row][ix][f] += dL / d values[row][ix][f].  Each contribution is a
 * forward-mode derivative seeded on one knot that the evaluation read.
 * Points with a NaN value contribute nothing.  gabs (may be NULL) receives
 * the sum of the contributions' magnitudes, the scale of the sum's rounding.
 * Serial. */
void og_knot_grad(const og *g, const double *x, const double *q2, long n, const double *cot,
                  double *gvals, double *gabs) {
  int rec[2 * 512];
  for (long p = 0; p < n; p++) {
    for (int f = 0; f < g->nf; f++) {
      double w = cot[p * g->nf + f];
      ctx c; memset(&c, 0, sizeof c); c.rec = rec;
      num r = xf_one(g, x[p], q2[p], f, &c);
      if (!isfinite(r.v)) continue;
      int nrec = c.nrec;
      for (int k = 0; k < nrec; k++) {
        ctx s; memset(&s, 0, sizeof s);
        s.wrt = WRT_KNOT; s.row = rec[2 * k]; s.ix = rec[2 * k + 1];
        double d = xf_one(g, x[p], q2[p], f, &s).d;
        gvals[((size_t)s.row * g->nx + s.ix) * g->nf + f] += w * d;
        if (gabs) gabs[((size_t)s.row * g->nx + s.ix) * g->nf + f] += fabs(w * d);
      }
    }
  }
}

/* The knots (row, ix) whose values one evaluation reads; returns how many. */
int og_knots_read(const og *g, double x, double q2, int f, int *rows_ix, int cap) {
  int rec[2 * 512];
  ctx c; memset(&c, 0, sizeof c); c.rec = rec;
  xf_one(g, x, q2, f, &c);
  int n = c.nrec < cap ? c.nrec : cap;
  memcpy(rows_ix, rec, sizeof(int) * 2 * n);
  return c.nrec;
}

void og_alphas(const og *g, const double *q2, long n, double *out_v, double *out_s, double *out_d,
               int nthreads) {
#pragma omp parallel for schedule(static) num_threads(threads(nthreads))
  for (long p = 0; p < n; p++) {
    num r = alphas_one(g, q2[p], out_d != NULL);
    out_v[p] = r.v;
    if (out_s) out_s[p] = r.s;
    if (out_d) out_d[p] = r.d;
  }
}

/* The bare Hermite segment, exposed for the cubic-exactness pin. */
double og_hermite(double t, double f0, double f1, double m0, double m1) {
  return hermite(cst(t), cst(1.0 - t), cst(f0), cst(f1), cst(m0), cst(m1)).v;
}

int og_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
