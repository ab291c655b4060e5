// grid.cu -- pdf_load_grid: validation, device layout and staging kernels.
//
// Staging (PDFFlow Sec. 2.2, the LHAPDF data loaded once into device
// memory) precomputes everything that depends only on the grid:
//   - ln of every knot (the evaluation kernels' own table-driven logarithm,
//     so a query on a knot gets t = 0 exactly);
//   - per cell, the tangent-augmented Hermite weights w_a(t) as cubics: the
//     knot tangent is the mean of the two adjacent secant slopes, one-sided
//     at the x edges and at the ends of each Q subgrid (Sec. 2.2's special
//     care at edges and thresholds), times the cell width;
//   - per cell and flavour, the bicubic patch sum_ab w_a(t) w_b(u) f_ab as
//     its 4x4 Bezier control points (Bernstein basis), in FP64 and rounded
//     to FP32;
//   - per alpha_s cell the cubic in u in monomial form (Sec. 2.3; one
//     dimension, four well-scaled coefficients), same tangents per subgrid;
//   - a degenerate cell on the last x knot and on the top Q knot (t = 0
//     there; its patch carries only that knot's column or row), so the last
//     knots are reproduced exactly;
//   - fixed sites used by the continuation (1.01 Q2min, the top knots) and
//     float thresholds for the exact FP32 search.
#include <atomic>
#include <cmath>
#include <vector>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <new>

#include "ffmath.cuh"
#include "pdf_internal.cuh"

namespace pdfgb {

static thread_local char g_errbuf[512];

int set_error(int code, const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_errbuf, sizeof g_errbuf, fmt, ap);
  va_end(ap);
  return code;
}

int check_launch(const char *what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(PDF_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
  return PDF_OK;
}

std::atomic<size_t> g_scratch_limit{SIZE_MAX};
size_t scratch_limit() { return g_scratch_limit.load(std::memory_order_relaxed); }

// Stream-ordered scratch of the sorted paths, from a pool of the device's
// own (kept between calls up to 256 MB, so a call does not map memory afresh).
cudaMemPool_t sort_pool(int dev) {
  static std::mutex mu;
  static cudaMemPool_t pools[64] = {};
  if (dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> lock(mu);
  if (!pools[dev]) {
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t p = nullptr;
    if (cudaMemPoolCreate(&p, &props) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    unsigned long long keep = 256ull << 20;
    cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep);
    pools[dev] = p;
  }
  return pools[dev];
}

// Knot weights of one cell in the cubic Bernstein basis
// B_k(t) = C(3,k) t^k (1-t)^(3-k):  w_a(t) = sum_k W[a][k] B_k(t) is the
// weight of knot i-1+a.  A cubic Hermite segment with end values f_i, f_{i+1}
// and end tangents m0, m1 (slope times cell width d) has the Bezier control
// points f_i, f_i + m0/3, f_{i+1} - m1/3, f_{i+1}.  The tangents are the
// finite differences of Sec. 2.2: at the left knot m0 = aL (f_{i+1} - f_i) +
// bm (f_i - f_{i-1}), at the right knot m1 = dR (f_{i+1} - f_i) +
// gp (f_{i+2} - f_{i+1}); inside the grid aL = dR = 1/2, bm = d/(2 d_prev),
// gp = d/(2 d_next); at an edge the one-sided secant (aL = 1, bm = 0 or
// dR = 1, gp = 0).  Bernstein weights are non-negative and sum to one, so a
// patch evaluated in this basis suffers no cancellation.
__device__ void cell_weights(double aL, double bm, double dR, double gp, double *W) {
  const double third = 1.0 / 3.0;
  double V[4][4] = {{0.0, 1.0, 0.0, 0.0},
                    {-bm * third, 1.0 + (bm - aL) * third, aL * third, 0.0},
                    {0.0, dR * third, 1.0 - (dR - gp) * third, -gp * third},
                    {0.0, 0.0, 1.0, 0.0}};  // V[k][a]
  for (int a = 0; a < 4; a++)
    for (int k = 0; k < 4; k++) W[a * 4 + k] = V[k][a];
}

struct Stage {
  // inputs (device copies)
  const double *xk, *q2k, *vals, *aq2, *aval;
  const int *first, *nq;
  int nx, nrows, nf, na, nsub, nxc, nqc;
  int nfp;   // flavour stride of the FP32 and float-float copies (nf rounded up to 8)
  int nmem;  // members: values and control points repeat per member
  // outputs
  double *lx, *lq, *alq;
  double *xcell, *qcell, *xW, *qW, *coef, *acell;
  float *coef32, *xthr32, *q2thr32, *aq2thr32, *xcell32, *qcell32, *acell32;
  float2 *coefff;
  double2 *tlogtab;  // tang.cuh tables, filled on the host before staging
  double *tloghtab, *texptab;
  float4 *fflog;     // ffmath.cuh tables, likewise
  float2 *ffexp;
  float4 *xposff, *qposff, *aposff, *lnfff;  // ffpos.cuh tables, likewise
  float2 *lnfff2;
  int *ffbad;  // set when a control point is outside the float-float range
  int *row_qc, *qc_row;
  double *scal;  // scalar outputs, see k_scalars
};

__global__ void k_logs(Stage S) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  const LogTabs LT{S.tlogtab, S.tloghtab};
  if (i < S.nx) { S.lx[i] = tlog(S.xk[i], LT); S.xthr32[i] = __double2float_ru(S.xk[i]); }
  if (i < S.nrows) { S.lq[i] = tlog(S.q2k[i], LT); S.q2thr32[i] = __double2float_ru(S.q2k[i]); }
  if (i < S.na) { S.alq[i] = tlog(S.aq2[i], LT); S.aq2thr32[i] = __double2float_ru(S.aq2[i]); }
}

void tang_tables(double *logtab, double *loghtab, double *exptab) {
  for (int j = 0; j < kLogTab; j++) {
    const double F = 1.0 + j / 256.0;
    logtab[2 * j] = 1.0 / F;
    logtab[2 * j + 1] = j == kLogTab - 1 ? kLn2 : (double)logl((long double)F);
    loghtab[j] = (double)logl((long double)F / 2.0L);
  }
  for (int k = 0; k < kExpTab; k++) exptab[k] = (double)exp2l((long double)k / 256.0L);
}

// Float-float tables of ffmath.cuh: c_j = 1/F_j rounded to float and -ln c_j
// split into hi + lo (F_j = 1 + j/128), and 2^(k/64) split likewise.
void ff_tables(float *logtab, float *exptab) {
  auto split = [](long double v, float *o) {
    o[0] = (float)v;
    o[1] = (float)(v - (long double)o[0]);
  };
  for (int j = 0; j < kFFLogTab; j++) {
    const float c = (float)(1.0L / (1.0L + j / 128.0L));
    logtab[4 * j] = c;
    split(-logl((long double)c), logtab + 4 * j + 1);
    logtab[4 * j + 3] = 0.f;
  }
  for (int k = 0; k < kFFExpTab; k++) split(exp2l(k / 64.0L), exptab + 2 * k);
}

// ffpos.cuh tables.  A knot a starting a cell that ends at b (b = a: no
// cell): {ln m hi, lo, 1/ln(b/a) hi, lo}, with a = 2^e m and m taken in
// [sqrt(1/2), sqrt(2)) by the device's test on the bits (ff_sig_high).
static float4 pos_entry(double a, double b) {
  long long bits;
  std::memcpy(&bits, &a, sizeof bits);
  const bool high = ((bits >> 32) & 0xFFFFF) >= 0x6A09E;
  int e2 = 0;
  long double m = 2.0L * frexpl((long double)a, &e2);  // [1, 2)
  if (high) m /= 2.0L;                                 // [sqrt(1/2), 1)
  const long double lm = logl(m);
  const long double id = b > a ? 1.0L / logl((long double)b / (long double)a) : 0.0L;
  float4 r;
  r.x = (float)lm;
  r.y = (float)(lm - (long double)r.x);
  r.z = (float)id;
  r.w = (float)(id - (long double)r.z);
  return r;
}
// {1/F_j hi, lo, ln F_j hi, lo} and ln(F_j / 2) {hi, lo} for F_j = 1 + j/256,
// j = 0..256 (tang.cuh's steps)
static void ln_f_table(float4 *o, float2 *o2) {
  for (int j = 0; j < kLogTab; j++) {
    const long double F = 1.0L + j / 256.0L, iF = 1.0L / F, lF = logl(F), lF2 = logl(F / 2.0L);
    o[j].x = (float)iF;
    o[j].y = (float)(iF - (long double)o[j].x);
    o[j].z = (float)lF;
    o[j].w = (float)(lF - (long double)o[j].z);
    o2[j].x = (float)lF2;
    o2[j].y = (float)(lF2 - (long double)o2[j].x);
  }
}

// FP32 cell table: both end knots rounded to float (k0f, k1f), their float
// reciprocals, the FP64 corrections ln(kf / k) that undo the rounding, the
// inverse cell width in ln, and the geometric midpoint that picks the nearer
// end as the reference of the logarithm:
//   {k0f, 1/k0f, ln(k0f/k0), 1/d, k1f, 1/k1f, ln(k1f/k1), mid}.
__device__ void cell32(double k0, double k1, double inv_d, double mid, float *o) {
  float k0f = (float)k0, k1f = (float)k1;
  o[0] = k0f; o[1] = (float)(1.0 / (double)k0f); o[2] = (float)log((double)k0f / k0); o[3] = (float)inv_d;
  o[4] = k1f; o[5] = (float)(1.0 / (double)k1f); o[6] = (float)log((double)k1f / k1); o[7] = (float)mid;
}

// Degenerate cell on a last knot: all weight on the knot itself (a = 1),
// whatever t (every Bernstein coefficient of w_1 is one).
__device__ void knot_weights(double *W) {
  for (int m = 0; m < 16; m++) W[m] = 0.0;
  for (int k = 0; k < 4; k++) W[1 * 4 + k] = 1.0;
}

__global__ void k_xcells(Stage S) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= S.nx) return;
  if (i == S.nx - 1) {  // {ln x_i, 0, ln x_i, 1}: t = 0 and 1 - t = 1 exactly
    S.xcell[4 * i] = S.lx[i];
    S.xcell[4 * i + 1] = 0.0;
    S.xcell[4 * i + 2] = S.lx[i];
    S.xcell[4 * i + 3] = 1.0;
    cell32(S.xk[i], S.xk[i], 0.0, INFINITY, S.xcell32 + 8 * i);
    knot_weights(S.xW + 16 * i);
    return;
  }
  double d = S.lx[i + 1] - S.lx[i];
  S.xcell[4 * i] = S.lx[i];
  S.xcell[4 * i + 1] = 1.0 / d;
  S.xcell[4 * i + 2] = S.lx[i + 1];
  S.xcell[4 * i + 3] = 0.0;
  cell32(S.xk[i], S.xk[i + 1], 1.0 / d, sqrt(S.xk[i] * S.xk[i + 1]), S.xcell32 + 8 * i);
  double aL = 1.0, bm = 0.0, dR = 1.0, gp = 0.0;
  if (i > 0) { aL = 0.5; bm = 0.5 * d / (S.lx[i] - S.lx[i - 1]); }
  if (i + 1 < S.nx - 1) { dR = 0.5; gp = 0.5 * d / (S.lx[i + 2] - S.lx[i + 1]); }
  cell_weights(aL, bm, dR, gp, S.xW + 16 * i);
}

__global__ void k_qcells(Stage S) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= S.nrows) return;
  int s = 0, qc0 = 0;
  while (s + 1 < S.nsub && j >= S.first[s + 1]) { qc0 += S.nq[s] - 1; s++; }
  int j0 = S.first[s], j1 = S.first[s] + S.nq[s] - 1;
  if (j == S.nrows - 1) {  // top knot: degenerate cell nqc
    S.row_qc[j] = S.nqc;
    S.qc_row[S.nqc] = j;
    S.qcell[4 * j] = S.lq[j];
    S.qcell[4 * j + 1] = 0.0;
    S.qcell[4 * j + 2] = S.lq[j];
    S.qcell[4 * j + 3] = 1.0;
    cell32(S.q2k[j], S.q2k[j], 0.0, INFINITY, S.qcell32 + 8 * j);
    knot_weights(S.qW + 16 * S.nqc);
    return;
  }
  if (j >= j1) {  // last row of a lower subgrid starts no cell
    S.row_qc[j] = -1;
    for (int m = 0; m < 4; m++) S.qcell[4 * j + m] = 0.0;
    return;
  }
  int qc = qc0 + (j - j0);
  S.row_qc[j] = qc;
  S.qc_row[qc] = j;
  double d = S.lq[j + 1] - S.lq[j];
  S.qcell[4 * j] = S.lq[j];
  S.qcell[4 * j + 1] = 1.0 / d;
  S.qcell[4 * j + 2] = S.lq[j + 1];
  S.qcell[4 * j + 3] = 0.0;
  cell32(S.q2k[j], S.q2k[j + 1], 1.0 / d, sqrt(S.q2k[j] * S.q2k[j + 1]), S.qcell32 + 8 * j);
  double aL = 1.0, bm = 0.0, dR = 1.0, gp = 0.0;
  if (j > j0) { aL = 0.5; bm = 0.5 * d / (S.lq[j] - S.lq[j - 1]); }
  if (j + 1 < j1) { dR = 0.5; gp = 0.5 * d / (S.lq[j + 2] - S.lq[j + 1]); }
  cell_weights(aL, bm, dR, gp, S.qW + 16 * qc);
}

// One thread per (member, q cell, x cell, flavour) slot, degenerate ones
// included: control point b[l][k] = sum_ab W_x[a][k] W_q[b][l] f_ab.
__global__ void k_coef(Stage S) {
  long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long per = (long long)(S.nqc + 1) * S.nx * S.nf;
  if (gid >= per * (S.nmem > 0 ? S.nmem : 1)) return;
  const long long mem = gid / per, id = gid - mem * per;
  const double *vals = S.vals + mem * (long long)S.nrows * S.nx * S.nf;
  int f = (int)(id % S.nf);
  long long cell = id / S.nf;
  int xc = (int)(cell % S.nx), qc = (int)(cell / S.nx);
  int j = S.qc_row[qc], i = xc;
  const double *Wx = S.xW + 16 * xc, *Wq = S.qW + 16 * qc;
  double c[16];
  for (int m = 0; m < 16; m++) c[m] = 0.0;
  for (int b = 0; b < 4; b++) {
    int row = j - 1 + b;
    if (row < 0 || row >= S.nrows) continue;
    for (int a = 0; a < 4; a++) {
      int col = i - 1 + a;
      if (col < 0 || col >= S.nx) continue;
      double fv = vals[((size_t)row * S.nx + col) * S.nf + f];
      for (int l = 0; l < 4; l++) {
        double wl = Wq[b * 4 + l] * fv;
        for (int k = 0; k < 4; k++) c[l * 4 + k] = fma(Wx[a * 4 + k], wl, c[l * 4 + k]);
      }
    }
  }
  double *o = S.coef + (size_t)gid * 16;
  // FP32 copy row-major by control-point row, then flavour: [cell][l][f][4], so
  // one load instruction over the flavours of a point reads consecutive rows;
  // the flavour stride nfp (a multiple of 8) makes each row block whole lines
  float *o32 = S.coef32 + (size_t)(gid / S.nf) * 16 * S.nfp + (size_t)f * 4;
  // float-float copy flavour-minor by pairs of control points,
  // [cell][m / 2][flavour][4] = {hi_m, hi_m+1, lo_m, lo_m+1} (m even): one
  // 16-byte load per pair and flavour, the lanes of one load (consecutive
  // flavours of a point) read consecutive bytes, and the two high (low) parts
  // land in one register pair for packed f32x2 arithmetic
  float *off = reinterpret_cast<float *>(S.coefff + (size_t)(gid / S.nf) * 16 * S.nfp) + (size_t)f * 4;
  bool bad = false;
  for (int m = 0; m < 16; m++) {
    o[m] = c[m];
    o32[(size_t)(m >> 2) * 4 * S.nfp + (m & 3)] = (float)c[m];
    // float-float split: hi = round(c), lo = round(c - hi); exact to 2^-48 of c
    // while |c| stays well inside the float exponent range
    float hi = __double2float_rn(c[m]);
    float lo = __double2float_rn(c[m] - (double)hi);
    off[(size_t)(m >> 1) * 4 * S.nfp + (m & 1)] = hi;
    off[(size_t)(m >> 1) * 4 * S.nfp + 2 + (m & 1)] = lo;
    double a = fabs(c[m]);
    if (a != 0.0 && (a < 1e-30 || a > 1e30)) bad = true;
  }
  if (bad && S.ffbad) atomicOr(S.ffbad, 1);
}

// alpha_s cells: one thread per node; the last node gets a degenerate cell.
__global__ void k_acells(Stage S) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= S.na) return;
  double *o = S.acell + 6 * k;
  float *o32 = S.acell32 + 6 * k;
  if (k == S.na - 1) {
    o[0] = S.alq[k]; o[1] = 0.0; o[2] = S.aval[k]; o[3] = o[4] = o[5] = 0.0;
    o32[0] = (float)(1.0 / S.aq2[k]); o32[1] = 0.f; o32[2] = (float)S.aval[k];
    o32[3] = o32[4] = o32[5] = 0.f;
    return;
  }
  if (!(S.aq2[k] < S.aq2[k + 1])) {  // zero-width pair at a threshold: not a cell
    for (int m = 0; m < 6; m++) { o[m] = 0.0; o32[m] = 0.f; }
    return;
  }
  const double *l = S.alq, *f = S.aval;
  double d = l[k + 1] - l[k];
  bool left_edge = (k == 0) || (S.aq2[k] == S.aq2[k - 1]);
  bool right_edge = (k + 1 == S.na - 1) || (S.aq2[k + 2] == S.aq2[k + 1]);
  double sec = (f[k + 1] - f[k]) / d;
  double s0 = left_edge ? sec : 0.5 * (sec + (f[k] - f[k - 1]) / (l[k] - l[k - 1]));
  double s1 = right_edge ? sec : 0.5 * (sec + (f[k + 2] - f[k + 1]) / (l[k + 2] - l[k + 1]));
  double m0 = d * s0, m1 = d * s1;
  o[0] = l[k];
  o[1] = 1.0 / d;
  o[2] = f[k];
  o[3] = m0;
  o[4] = -3.0 * f[k] + 3.0 * f[k + 1] - 2.0 * m0 - m1;
  o[5] = 2.0 * f[k] - 2.0 * f[k + 1] + m0 + m1;
  o32[0] = (float)(1.0 / S.aq2[k]);
  o32[1] = (float)(1.0 / d);
  for (int m = 2; m < 6; m++) o32[m] = (float)o[m];
}

// Scalars (single thread).  scal layout:
//  2 top_qc  3 q101_qc  4 q101_u  5 lx0  6 idx0  7 lq2max  8 idq_top  9 ln101
__global__ void k_scalars(Stage S) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double *o = S.scal;
  int top = S.nrows - 2;
  o[2] = (double)S.row_qc[top];
  double v = 1.01 * S.q2k[0];
  int j = 0;  // same rule as the query search: the last row with Q^2_j <= v
  while (j + 1 < S.nrows && S.q2k[j + 1] <= v) j++;
  o[3] = (double)S.row_qc[j];
  const LogTabs LT{S.tlogtab, S.tloghtab};
  o[4] = (tlog(v, LT) - S.qcell[4 * j]) * S.qcell[4 * j + 1];
  o[5] = S.xcell[0];
  o[6] = S.xcell[1];
  o[7] = S.lq[S.nrows - 1];
  o[8] = S.qcell[4 * top + 1];
  o[9] = tlog(1.01, LT);
}

static int pow2_floor(int n) {
  int p = 1;
  while (p * 2 <= n) p *= 2;
  return n >= 1 ? p : 0;
}

static int validate(const pdf_grid_desc *d, int *nrows_out) {
  if (!d) return set_error(PDF_ERR_NULL, "pdf_load_grid: descriptor is NULL");
  if (!d->x_knots || !d->nq || !d->q2_knots || !d->pids || !d->values)
    return set_error(PDF_ERR_NULL, "pdf_load_grid: a descriptor array is NULL");
  if (d->nx < 2 || d->nx > PDF_MAX_NX)
    return set_error(PDF_ERR_GRID, "pdf_load_grid: nx = %d outside [2, %d]", d->nx, PDF_MAX_NX);
  if (d->nflav < 1 || d->nflav > PDF_MAX_NFLAV)
    return set_error(PDF_ERR_GRID, "pdf_load_grid: nflav = %d outside [1, %d]", d->nflav, PDF_MAX_NFLAV);
  if (d->nsub < 1) return set_error(PDF_ERR_GRID, "pdf_load_grid: nsub = %d < 1", d->nsub);
  for (int i = 0; i < d->nx; i++) {
    double x = d->x_knots[i];
    if (!(x > 0.0) || !(x <= 1.0))
      return set_error(PDF_ERR_GRID, "pdf_load_grid: x knot %d = %g outside (0, 1]", i, x);
    if (i > 0 && !(x > d->x_knots[i - 1]))
      return set_error(PDF_ERR_GRID, "pdf_load_grid: x knots not strictly increasing at %d", i);
  }
  long rows = 0;
  for (int s = 0; s < d->nsub; s++) {
    if (d->nq[s] < 2) return set_error(PDF_ERR_GRID, "pdf_load_grid: subgrid %d has %d < 2 knots", s, d->nq[s]);
    rows += d->nq[s];
    if (rows > PDF_MAX_ROWS) return set_error(PDF_ERR_GRID, "pdf_load_grid: more than %d Q rows", PDF_MAX_ROWS);
  }
  int r0 = 0;
  for (int s = 0; s < d->nsub; s++) {
    for (int j = r0; j < r0 + d->nq[s]; j++) {
      double q = d->q2_knots[j];
      if (!(q > 0.0) || !std::isfinite(q))
        return set_error(PDF_ERR_GRID, "pdf_load_grid: Q2 knot %d = %g not positive and finite", j, q);
      if (j > r0 && !(q > d->q2_knots[j - 1]))
        return set_error(PDF_ERR_GRID, "pdf_load_grid: Q2 knots of subgrid %d not strictly increasing", s);
    }
    if (s > 0 && d->q2_knots[r0] != d->q2_knots[r0 - 1])
      return set_error(PDF_ERR_GRID, "pdf_load_grid: subgrid %d does not start at the previous one's last knot", s);
    r0 += d->nq[s];
  }
  if (!(d->q2_knots[rows - 1] >= 1.01 * d->q2_knots[0]))
    return set_error(PDF_ERR_GRID, "pdf_load_grid: Q2 range narrower than a factor 1.01");
  size_t nv = (size_t)rows * d->nx * d->nflav;
  for (size_t k = 0; k < nv; k++)
    if (!std::isfinite(d->values[k])) return set_error(PDF_ERR_GRID, "pdf_load_grid: value %zu not finite", k);
  for (int f = 0; f < d->nflav; f++)
    for (int g = 0; g < f; g++)
      if (d->pids[f] == d->pids[g]) return set_error(PDF_ERR_GRID, "pdf_load_grid: pid %d repeated", d->pids[f]);
  if (d->na < 0 || d->na == 1 || d->na > PDF_MAX_NALPHAS)
    return set_error(PDF_ERR_GRID, "pdf_load_grid: na = %d (0, or 2..%d)", d->na, PDF_MAX_NALPHAS);
  if (d->na > 0) {
    if (!d->as_q2 || !d->as_vals) return set_error(PDF_ERR_NULL, "pdf_load_grid: alpha_s arrays NULL");
    int run = 1;
    for (int k = 0; k < d->na; k++) {
      if (!(d->as_q2[k] > 0.0) || !std::isfinite(d->as_q2[k]) || !std::isfinite(d->as_vals[k]))
        return set_error(PDF_ERR_GRID, "pdf_load_grid: alpha_s node %d invalid", k);
      if (k > 0) {
        if (d->as_q2[k] < d->as_q2[k - 1])
          return set_error(PDF_ERR_GRID, "pdf_load_grid: alpha_s nodes decrease at %d", k);
        if (d->as_q2[k] == d->as_q2[k - 1]) {
          if (run < 2) return set_error(PDF_ERR_GRID, "pdf_load_grid: alpha_s subgrid with < 2 nodes");
          run = 1;
        } else {
          run++;
        }
      }
    }
    if (run < 2) return set_error(PDF_ERR_GRID, "pdf_load_grid: alpha_s subgrid with < 2 nodes");
  }
  *nrows_out = (int)rows;
  return PDF_OK;
}

// Bump allocator over one device allocation.
struct Arena {
  char *base = nullptr;
  size_t off = 0, cap = 0;
  template <typename T>
  T *take(size_t count) {
    size_t bytes = ((count * sizeof(T) + 255) / 256) * 256;
    T *p = reinterpret_cast<T *>(base + off);
    off += bytes;
    return p;
  }
};

}  // namespace pdfgb

using namespace pdfgb;

extern "C" const char *pdf_last_error(void) { return g_errbuf; }

extern "C" int pdf_set_scratch_limit(size_t bytes) {
  g_scratch_limit.store(bytes, std::memory_order_relaxed);
  return PDF_OK;
}
extern "C" int pdf_get_scratch_limit(size_t *bytes) {
  if (!bytes) return set_error(PDF_ERR_NULL, "pdf_get_scratch_limit: NULL output");
  *bytes = scratch_limit();
  return PDF_OK;
}

static int load_impl(const pdf_grid_desc *d, int nmem, const double *member_values, pdf_grid **out) {
  g_errbuf[0] = 0;
  if (!out) return set_error(PDF_ERR_NULL, "pdf_load_grid: out is NULL");
  *out = nullptr;
  if (!d) return set_error(PDF_ERR_NULL, "pdf_load_grid: descriptor is NULL");
  pdf_grid_desc dd = *d;  // a member set is validated on its first member
  if (member_values) dd.values = member_values;
  int nrows = 0;
  int rc = validate(&dd, &nrows);
  if (rc) return rc;
  d = &dd;
  if (nmem < 1) return set_error(PDF_ERR_ARG, "pdf_load_grid_members: nmem = %d < 1", nmem);
  if (member_values) {
    size_t nv = (size_t)nmem * nrows * d->nx * d->nflav;
    for (size_t k = 0; k < nv; k++)
      if (!std::isfinite(member_values[k])) return set_error(PDF_ERR_GRID, "pdf_load_grid_members: value %zu not finite", k);
  }
  const double *values0 = member_values ? member_values : d->values;
  const int nx = d->nx, nf = d->nflav, na = d->na, nsub = d->nsub;
  const int nxc = nx - 1, nqc = nrows - nsub;
  const int nfp = (nf + 7) & ~7;

  // sizes (a dry run of the arena)
  auto layout = [&](Arena &A, Stage &S, unsigned long long **inv) {
    S.xk = A.take<double>(nx); S.q2k = A.take<double>(nrows);
    S.vals = A.take<double>((size_t)nmem * nrows * nx * nf);
    S.aq2 = A.take<double>(na > 0 ? na : 1); S.aval = A.take<double>(na > 0 ? na : 1);
    S.first = A.take<int>(nsub); S.nq = A.take<int>(nsub);
    S.lx = A.take<double>(nx); S.lq = A.take<double>(nrows); S.alq = A.take<double>(na > 0 ? na : 1);
    S.xcell = A.take<double>(4 * nx); S.qcell = A.take<double>(4 * nrows);
    S.xW = A.take<double>(16 * nx); S.qW = A.take<double>(16 * (nqc + 1));
    S.coef = A.take<double>((size_t)nmem * (nqc + 1) * nx * nf * 16);
    S.coef32 = A.take<float>((size_t)nmem * (nqc + 1) * nx * nfp * 16);
    S.coefff = A.take<float2>((size_t)nmem * (nqc + 1) * nx * nfp * 16);
    S.ffbad = A.take<int>(1);
    S.tlogtab = A.take<double2>(kLogTab); S.tloghtab = A.take<double>(kLogTab);
    S.texptab = A.take<double>(kExpTab);
    S.fflog = A.take<float4>(kFFLogTab); S.ffexp = A.take<float2>(kFFExpTab);
    S.xposff = A.take<float4>(nx); S.qposff = A.take<float4>(nrows);
    S.aposff = A.take<float4>(na > 0 ? na : 1); S.lnfff = A.take<float4>(kLogTab);
    S.lnfff2 = A.take<float2>(kLogTab);
    S.acell = A.take<double>(6 * (na > 0 ? na : 1));
    S.acell32 = A.take<float>(6 * (na > 0 ? na : 1));
    S.xthr32 = A.take<float>(nx); S.q2thr32 = A.take<float>(nrows); S.aq2thr32 = A.take<float>(na > 0 ? na : 1);
    S.xcell32 = A.take<float>(8 * nx); S.qcell32 = A.take<float>(8 * nrows);
    S.row_qc = A.take<int>(nrows); S.qc_row = A.take<int>(nqc + 1);
    S.scal = A.take<double>(16);
    *inv = A.take<unsigned long long>(1);
  };
  Arena dry;
  Stage S{};
  unsigned long long *inv = nullptr;
  layout(dry, S, &inv);

  pdf_grid *g = new (std::nothrow) pdf_grid();
  if (!g) return set_error(PDF_ERR_ALLOC, "pdf_load_grid: host allocation failed");
  cudaGetDevice(&g->device);
  void *base = nullptr;
  cudaError_t e = cudaMalloc(&base, dry.off);
  if (e != cudaSuccess) {
    delete g;
    return set_error(PDF_ERR_ALLOC, "pdf_load_grid: cudaMalloc(%zu): %s", dry.off, cudaGetErrorString(e));
  }
  g->blocks[0] = base;
  g->nblocks = 1;
  Arena A;
  A.base = static_cast<char *>(base);
  A.cap = dry.off;
  layout(A, S, &inv);
  S.nx = nx; S.nrows = nrows; S.nf = nf; S.na = na; S.nsub = nsub; S.nxc = nxc; S.nqc = nqc;
  S.nfp = nfp;
  S.nmem = nmem;

  int first[1024];
  for (int s = 0, r = 0; s < nsub; s++) { first[s] = r; r += d->nq[s]; }
  auto H2D = [&](const void *dst, const void *src, size_t bytes) {
    if (e == cudaSuccess && bytes) e = cudaMemcpy(const_cast<void *>(dst), src, bytes, cudaMemcpyHostToDevice);
  };
  H2D(S.xk, d->x_knots, sizeof(double) * nx);
  H2D(S.q2k, d->q2_knots, sizeof(double) * nrows);
  H2D(S.vals, values0, sizeof(double) * (size_t)nmem * nrows * nx * nf);
  if (na > 0) { H2D(S.aq2, d->as_q2, sizeof(double) * na); H2D(S.aval, d->as_vals, sizeof(double) * na); }
  H2D(S.first, first, sizeof(int) * nsub);
  H2D(S.nq, d->nq, sizeof(int) * nsub);
  {
    double lt[2 * kLogTab], lh[kLogTab], et[kExpTab];
    tang_tables(lt, lh, et);
    H2D(S.tlogtab, lt, sizeof lt);
    H2D(S.tloghtab, lh, sizeof lh);
    H2D(S.texptab, et, sizeof et);
    float fl[4 * kFFLogTab], fe[2 * kFFExpTab];
    ff_tables(fl, fe);
    H2D(S.fflog, fl, sizeof fl);
    H2D(S.ffexp, fe, sizeof fe);
  }
  // Member sets keep the FP64 logarithm for positions: their kernel repeats
  // the per-point work for every chunk of members with about two units per
  // warp, so the warps run it in step and its longer float-float dependency
  // chain is not hidden (400 members x 2415 points: 0.234 against 0.193 ms).
  int ffpos = nmem > 1 ? 0 : 1;
  {
    std::vector<float4> xp(nx), qp(nrows), ap(na > 0 ? na : 1), lf(kLogTab);
    std::vector<float2> lf2(kLogTab);
    // a knot's row for each knot list; starts[k]: knot k starts a cell
    auto fill = [&](const double *k, int n, const std::vector<char> &starts, std::vector<float4> &o) {
      for (int i = 0; i < n; i++) {
        if (!(std::fpclassify(k[i]) == FP_NORMAL)) ffpos = 0;
        const bool st = starts[i] && i + 1 < n && k[i + 1] > k[i];
        if (st && std::abs(std::ilogb(k[i + 1]) - std::ilogb(k[i])) >= 100) ffpos = 0;
        o[i] = pos_entry(k[i], st ? k[i + 1] : k[i]);
      }
    };
    std::vector<char> xs(nx, 1), qs(nrows, 0), as(na > 0 ? na : 1, 1);
    for (int s = 0; s < nsub; s++)
      for (int r = first[s]; r < first[s] + d->nq[s] - 1; r++) qs[r] = 1;
    fill(d->x_knots, nx, xs, xp);
    fill(d->q2_knots, nrows, qs, qp);
    if (na > 0) fill(d->as_q2, na, as, ap);
    ln_f_table(lf.data(), lf2.data());
    H2D(S.xposff, xp.data(), sizeof(float4) * nx);
    H2D(S.qposff, qp.data(), sizeof(float4) * nrows);
    if (na > 0) H2D(S.aposff, ap.data(), sizeof(float4) * na);
    H2D(S.lnfff, lf.data(), sizeof(float4) * kLogTab);
    H2D(S.lnfff2, lf2.data(), sizeof(float2) * kLogTab);
  }
  if (e == cudaSuccess) e = cudaMemset(inv, 0, sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMemset(S.ffbad, 0, sizeof(int));
  if (e != cudaSuccess) {
    pdf_free_grid(g);
    return set_error(PDF_ERR_CUDA, "pdf_load_grid: copy to device: %s", cudaGetErrorString(e));
  }

  int nmax = nx > nrows ? nx : nrows;
  if (na > nmax) nmax = na;
  k_logs<<<(nmax + 127) / 128, 128>>>(S);
  k_xcells<<<(nx + 127) / 128, 128>>>(S);
  k_qcells<<<(nrows + 127) / 128, 128>>>(S);
  long long ncoef = (long long)nmem * (nqc + 1) * nx * nf;
  k_coef<<<(unsigned)((ncoef + 127) / 128), 128>>>(S);
  if (na > 1) k_acells<<<(na + 127) / 128, 128>>>(S);
  k_scalars<<<1, 32>>>(S);
  if ((rc = check_launch("pdf_load_grid staging"))) { pdf_free_grid(g); return rc; }
  double scal[16];
  int ffbad = 1;
  e = cudaMemcpy(scal, S.scal, sizeof scal, cudaMemcpyDeviceToHost);  // synchronises
  if (e == cudaSuccess) e = cudaMemcpy(&ffbad, S.ffbad, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) {
    pdf_free_grid(g);
    return set_error(PDF_ERR_CUDA, "pdf_load_grid: staging: %s", cudaGetErrorString(e));
  }

  GridView &v = g->v;
  v.nx = nx; v.nrows = nrows; v.nf = nf; v.nxc = nxc; v.nqc = nqc; v.na = na; v.nsub = nsub;
  v.xstep = pow2_floor(nx - 1); v.qstep = pow2_floor(nrows - 1); v.astep = na > 1 ? pow2_floor(na - 1) : 0;
  v.xk = S.xk; v.q2k = S.q2k; v.xcell = S.xcell; v.qcell = S.qcell; v.row_qc = S.row_qc;
  v.qc_row = S.qc_row; v.vals = const_cast<double *>(S.vals);
  v.coef = S.coef; v.coef32 = S.coef32; v.xW = S.xW; v.qW = S.qW;
  v.coefff = S.coefff; v.ff = ffbad ? 0 : 1;
  v.tlogtab = S.tlogtab; v.tloghtab = S.tloghtab; v.texptab = S.texptab;
  v.fflog = S.fflog; v.ffexp = S.ffexp;
  v.xposff = S.xposff; v.qposff = S.qposff; v.aposff = S.aposff; v.lnfff = S.lnfff; v.lnfff2 = S.lnfff2;
  v.ffpos = ffpos;
  v.nmem = nmem;
  v.mstride = (size_t)(nqc + 1) * nx * nf * 16;
  v.nfp = nfp;
  v.mstride_ff = (size_t)(nqc + 1) * nx * nfp * 16;
  g->ffbad = S.ffbad;
  v.xthr32 = S.xthr32; v.q2thr32 = S.q2thr32; v.xcell32 = S.xcell32; v.qcell32 = S.qcell32;
  v.aq2 = S.aq2; v.acell = S.acell; v.acell32 = S.acell32; v.aq2thr32 = S.aq2thr32;
  v.as_lo = na > 0 ? d->as_vals[0] : NAN;
  v.as_hi = na > 0 ? d->as_vals[na - 1] : NAN;
  v.x0 = d->x_knots[0]; v.xlast = d->x_knots[nx - 1];
  v.q2min = d->q2_knots[0]; v.q2max = d->q2_knots[nrows - 1];
  v.aq2lo = na > 0 ? d->as_q2[0] : NAN; v.aq2hi = na > 0 ? d->as_q2[na - 1] : NAN;
  // float thresholds: x < x0 <=> x < round_up(x0) for a float x, etc.
  auto ru = [](double a) { float f = (float)a; if ((double)f < a) f = nextafterf(f, INFINITY); return f; };
  auto rd = [](double a) { float f = (float)a; if ((double)f > a) f = nextafterf(f, -INFINITY); return f; };
  v.x0_ru = ru(v.x0); v.xlast_rd = rd(v.xlast); v.q2min_ru = ru(v.q2min); v.q2max_rd = rd(v.q2max);
  v.aq2lo_ru = na > 0 ? ru(v.aq2lo) : NAN; v.aq2hi_rd = na > 0 ? rd(v.aq2hi) : NAN;
  v.as_lo32 = (float)v.as_lo; v.as_hi32 = (float)v.as_hi;
  v.top_qc = (int)scal[2]; v.q101_qc = (int)scal[3]; v.q101_u = scal[4];
  v.lx0 = scal[5]; v.idx0 = scal[6]; v.lq2max = scal[7]; v.idq_top = scal[8]; v.ln101 = scal[9];
  v.inv_q2min = 1.0 / v.q2min;
  v.x0inv32 = (float)(1.0 / v.x0); v.idx0_32 = (float)v.idx0;
  v.q2maxinv32 = (float)(1.0 / v.q2max); v.idq_top32 = (float)v.idq_top;
  v.q2min32 = (float)v.q2min; v.ln101_32 = (float)v.ln101;
  v.iln101 = 1.0 / v.ln101; v.iln101_32 = (float)(1.0 / v.ln101);
  {
    const long double il = 1.0L / logl(1.01L);
    v.iln101_ffh = (float)il;
    v.iln101_ffl = (float)(il - (long double)v.iln101_ffh);
  }
  v.q101_u32 = (float)v.q101_u;
  {
    auto split = [](double a, float &h, float &l) { h = (float)a; l = (float)(a - (double)h); };
    split(v.q101_u, v.q101ff[0], v.q101ff[1]);
    split(1.0 - v.q101_u, v.q101ff[2], v.q101ff[3]);
  }
  v.invalid = inv;
  for (int f = 0; f < nf; f++) g->pids[f] = d->pids[f];
  *out = g;
  return PDF_OK;
}

extern "C" int pdf_load_grid(const pdf_grid_desc *d, pdf_grid **out) { return load_impl(d, 1, nullptr, out); }

extern "C" int pdf_load_grid_members(const pdf_grid_desc *d, int nmem, const double *member_values,
                                     pdf_grid **out) {
  if (!member_values) return set_error(PDF_ERR_NULL, "pdf_load_grid_members: member_values is NULL");
  return load_impl(d, nmem, member_values, out);
}

extern "C" int pdf_grid_nmembers(const pdf_grid *g) { return g ? g->v.nmem : set_error(PDF_ERR_NULL, "grid is NULL"); }

extern "C" int pdf_free_grid(pdf_grid *g) {
  if (!g) return PDF_OK;
  for (int k = 0; k < pdf_grid::kIoStreams; k++) {
    if (g->io_stream[k]) { cudaStreamSynchronize(g->io_stream[k]); cudaStreamDestroy(g->io_stream[k]); }
    if (g->io_buf[k]) cudaFree(g->io_buf[k]);
  }
  if (g->mc_buf) cudaFree(g->mc_buf);
  if (g->mc_part) cudaFree(g->mc_part);
  for (int b = 0; b < g->nblocks; b++) cudaFree(g->blocks[b]);
  delete g;
  return PDF_OK;
}

extern "C" int pdf_grid_nflav(const pdf_grid *g) { return g ? g->v.nf : set_error(PDF_ERR_NULL, "grid is NULL"); }

extern "C" int pdf_grid_pid_column(const pdf_grid *g, int pid) {
  if (!g) return set_error(PDF_ERR_NULL, "grid is NULL");
  if (pid == 0) pid = 21;
  for (int f = 0; f < g->v.nf; f++)
    if (g->pids[f] == pid) return f;
  return -1;
}

extern "C" int pdf_grid_invalid_count(const pdf_grid *g, unsigned long long *count) {
  if (!g || !count) return set_error(PDF_ERR_NULL, "pdf_grid_invalid_count: NULL argument");
  cudaError_t e = cudaMemcpy(count, g->v.invalid, sizeof *count, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return set_error(PDF_ERR_CUDA, "pdf_grid_invalid_count: %s", cudaGetErrorString(e));
  return PDF_OK;
}

extern "C" int pdf_grid_set_values(pdf_grid *g, const double *values, cudaStream_t stream) {
  if (!g || !values) return set_error(PDF_ERR_NULL, "pdf_grid_set_values: NULL argument");
  const GridView &v = g->v;
  size_t bytes = (size_t)v.nrows * v.nx * v.nf * sizeof(double);
  cudaError_t e = cudaMemcpyAsync(v.vals, values, bytes, cudaMemcpyDeviceToDevice, stream);
  if (e != cudaSuccess) return set_error(PDF_ERR_CUDA, "pdf_grid_set_values: %s", cudaGetErrorString(e));
  Stage S{};
  S.nx = v.nx; S.nrows = v.nrows; S.nf = v.nf; S.nqc = v.nqc; S.nxc = v.nxc;
  S.nfp = v.nfp;
  S.nmem = 1;  // member 0
  S.vals = v.vals; S.qc_row = const_cast<int *>(v.qc_row);
  S.xW = const_cast<double *>(v.xW); S.qW = const_cast<double *>(v.qW);
  S.coef = const_cast<double *>(v.coef); S.coef32 = const_cast<float *>(v.coef32);
  S.coefff = const_cast<float2 *>(v.coefff);
  S.ffbad = g->ffbad;
  e = cudaMemsetAsync(g->ffbad, 0, sizeof(int), stream);
  if (e != cudaSuccess) return set_error(PDF_ERR_CUDA, "pdf_grid_set_values: %s", cudaGetErrorString(e));
  long long ncoef = (long long)(v.nqc + 1) * v.nx * v.nf;
  k_coef<<<(unsigned)((ncoef + 127) / 128), 128, 0, stream>>>(S);
  int rc = check_launch("pdf_grid_set_values");
  if (rc) return rc;
  // the float-float fast path stays on only if the new values allow it
  int bad = 1;
  e = cudaMemcpyAsync(&bad, g->ffbad, sizeof(int), cudaMemcpyDeviceToHost, stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess) return set_error(PDF_ERR_CUDA, "pdf_grid_set_values: %s", cudaGetErrorString(e));
  g->v.ff = bad ? 0 : 1;
  return PDF_OK;
}

extern "C" int pdf_grid_reset_invalid_count(pdf_grid *g) {
  if (!g) return set_error(PDF_ERR_NULL, "pdf_grid_reset_invalid_count: grid is NULL");
  cudaError_t e = cudaMemset(g->v.invalid, 0, sizeof(unsigned long long));
  if (e != cudaSuccess) return set_error(PDF_ERR_CUDA, "pdf_grid_reset_invalid_count: %s", cudaGetErrorString(e));
  return PDF_OK;
}
