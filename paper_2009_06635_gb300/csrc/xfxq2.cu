// xfxq2.cu -- FP32 evaluation kernel for x f(x, Q^2), the alpha_s kernel,
// and the C entry points of both precisions (FP64 evaluation: xf64.cu).
//
// One warp owns a tile of 32 query points (16 events in the Monte Carlo
// layout).  Each block first copies the grid's knot keys and its FP32 cell
// tables (x cells, Q cells, the row-to-cell map, alpha_s cells) into shared
// memory, so the per-point table reads of phase 1 stay off the global path.
// Phase 1 (lane = point): read x and Q^2 (coalesced), classify against the
// grid edges with exact float thresholds, search the cells on the raw bit
// patterns, record the Bernstein weights of the patch sites (one slot-major
// row per point) and the continuation parameters; points are ordered by
// class so that lanes of one instruction take the same branch.  Phase 2
// (lane = item (point, column), consecutive items are consecutive outputs):
// one lane evaluates a whole item, four float4 rows of the cell's control
// points against weights read as two 16-byte shared loads, so one
// instruction covers 32 items.  (A group of 16 lanes per point, so that one
// load instruction reads whole row blocks of two points, measured 7% slower
// at 1e7 points: fewer L1 wavefronts, more instructions.)
#include <cmath>
#include <type_traits>

#include "sites.cuh"

namespace pdfgb {

constexpr int kWarps = 8;
constexpr int kThreads = 32 * kWarps;

// Per-warp record of the points of one tile, by class-sorted slot.  Row W[s]
// holds Bx0 | Bx1 | Bq0 | Bq1 (16 floats), padded to 80 bytes so that the few
// slots one load instruction touches fall in different banks (and stay
// 16-byte aligned).
struct alignas(16) Rec32 {
  int cls[32], xc0[32], xc1[32], qc0[32], qc1[32];
  int cell0[32];     // float4 offset of the (qc0, xc0) control-point block in coef32
  long long ob[32];  // output offset of the point's first column
  float W[32][20];
  float px[32], pq[32], lr[32];
};

// One site: sum_l Bq_b[l] (sum_k Bx_a[k] b[l][k]), rounded as
// (p0 + p1) + (p2 + p3) with p_l = Bq_b[l] * (the row's dot product).
// q: the item's first row; rows are nf float4 apart.
__device__ __forceinline__ float site32(const float4 *q, int nf, const float *w, int a, int b) {
  const float4 bx = *reinterpret_cast<const float4 *>(w + 4 * a);
  const float4 bq = *reinterpret_cast<const float4 *>(w + 8 + 4 * b);
  const float bqv[4] = {bq.x, bq.y, bq.z, bq.w};
  float pl[4];
#pragma unroll
  for (int l = 0; l < 4; l++) {
    const float4 v = __ldg(q + (size_t)l * nf);
    float rr = bx.x * v.x;
    rr = fmaf(bx.y, v.y, rr);
    rr = fmaf(bx.z, v.z, rr);
    rr = fmaf(bx.w, v.w, rr);
    pl[l] = __fmul_rn(rr, bqv[l]);
  }
  return (pl[0] + pl[1]) + (pl[2] + pl[3]);
}

// One item: column col of the point in slot p (the same arithmetic for every
// column count, so one flavour alone and all flavours give identical bits).
__device__ __forceinline__ float eval_item32(const GridView &g, const Rec32 &R, int p, int col) {
  const float4 *cb = reinterpret_cast<const float4 *>(g.coef32) + col;
  const size_t stride = (size_t)g.nfp * 4;  // float4 per cell
  const float *w = R.W[p];
  auto F = [&](int a, int b) {
    int xc = a ? R.xc1[p] : R.xc0[p];
    int qc = b ? R.qc1[p] : R.qc0[p];
    return site32(cb + ((size_t)qc * g.nx + xc) * stride, g.nfp, w, a, b);
  };
  return combine<float>(R.cls[p], R.px[p], R.pq[p], R.lr[p], g.iln101_32, F);
}

// An in-grid item: one site, its block offset taken once per point (the
// same arithmetic as eval_item32's class switch gives for C_IN).
__device__ __forceinline__ float eval_in32(const GridView &g, const Rec32 &R, int p, int col) {
  const float4 *q = reinterpret_cast<const float4 *>(g.coef32) + R.cell0[p] + col;
  return site32(q, g.nfp, R.W[p], 0, 0);
}

// Write a point into its record slot.
__device__ __forceinline__ void store_point32(Rec32 &R, int slot, const PointSites<float> &ps, long long ob,
                                              const GridView &g) {
  R.cls[slot] = ps.cls;
  R.xc0[slot] = ps.xc0; R.xc1[slot] = ps.xc1; R.qc0[slot] = ps.qc0; R.qc1[slot] = ps.qc1;
  R.cell0[slot] = (ps.qc0 * g.nx + ps.xc0) * g.nfp * 4;
  R.ob[slot] = ob;
  R.px[slot] = ps.px; R.pq[slot] = ps.pq; R.lr[slot] = ps.lr;
  if (ps.cls == C_INVALID) return;
  float bx0[4], bx1[4], bq0[4], bq1[4];
  bernstein<float>(ps.t0, ps.ts0, bx0);
  bernstein<float>(ps.t1, 1.f - ps.t1, bx1);
  bernstein<float>(ps.u0, ps.us0, bq0);
  bernstein<float>(ps.u1, 1.f - ps.u1, bq1);
  float4 *row = reinterpret_cast<float4 *>(R.W[slot]);
  row[0] = make_float4(bx0[0], bx0[1], bx0[2], bx0[3]);
  row[1] = make_float4(bx1[0], bx1[1], bx1[2], bx1[3]);
  row[2] = make_float4(bq0[0], bq0[1], bq0[2], bq0[3]);
  row[3] = make_float4(bq1[0], bq1[1], bq1[2], bq1[3]);
}

// Byte offsets of the kernel's shared-memory regions (every region starts on
// a 16-byte boundary).
struct Smem32 {
  size_t xkeys, qkeys, akeys, xcell, qcell, rowqc, acell, recs, total;
};
__host__ __device__ inline Smem32 smem32_layout(const GridView &g) {
  Smem32 L;
  L.xkeys = 0;
  L.qkeys = L.xkeys + keys_bytes(g.nx, 4);
  L.akeys = L.qkeys + keys_bytes(g.nrows, 4);
  L.xcell = L.akeys + keys_bytes(g.na, 4);
  L.qcell = L.xcell + (size_t)32 * g.nx;
  L.rowqc = L.qcell + (size_t)32 * g.nrows;
  L.acell = L.rowqc + keys_bytes(g.nrows, 4);
  L.recs = L.acell + keys_bytes(6 * g.na, 4);
  L.total = L.recs + kWarps * sizeof(Rec32);
  return L;
}

// MODE_POINTS: points xa[n], qa[n]; out[n][ncol] for columns col0..col0+ncol-1;
//              as_out[n] (alpha_s) when not null.
// MODE_MC:     events xa[n] (x1), xb[n] (x2), Q^2 = x1 x2 s; out[n][2 nf + 1].
template <int MODE>
__global__ void __launch_bounds__(kThreads, 3)
k_xf32(GridView g, const float *__restrict__ xa, const float *__restrict__ qa, const float *__restrict__ xb,
       float s, long long n, int col0, int ncol, float *__restrict__ out, float *__restrict__ as_out) {
  extern __shared__ __align__(16) unsigned char smem[];
  const Smem32 L = smem32_layout(g);
  int *xkeys = reinterpret_cast<int *>(smem + L.xkeys);
  int *qkeys = reinterpret_cast<int *>(smem + L.qkeys);
  int *akeys = reinterpret_cast<int *>(smem + L.akeys);
  float *xcell = reinterpret_cast<float *>(smem + L.xcell);
  float *qcell = reinterpret_cast<float *>(smem + L.qcell);
  int *rowqc = reinterpret_cast<int *>(smem + L.rowqc);
  float *acell = reinterpret_cast<float *>(smem + L.acell);
  Rec32 *recs = reinterpret_cast<Rec32 *>(smem + L.recs);
  const bool want_as = MODE == MODE_MC || as_out;
  load_keys<float>(g, xkeys, 0);
  load_keys<float>(g, qkeys, 1);
  if (want_as) load_keys<float>(g, akeys, 2);
  for (int i = threadIdx.x; i < 2 * g.nx; i += blockDim.x)
    reinterpret_cast<float4 *>(xcell)[i] = __ldg(reinterpret_cast<const float4 *>(g.xcell32) + i);
  for (int i = threadIdx.x; i < 2 * g.nrows; i += blockDim.x)
    reinterpret_cast<float4 *>(qcell)[i] = __ldg(reinterpret_cast<const float4 *>(g.qcell32) + i);
  for (int i = threadIdx.x; i < g.nrows; i += blockDim.x) rowqc[i] = __ldg(g.row_qc + i);
  if (want_as)
    for (int i = threadIdx.x; i < 6 * g.na; i += blockDim.x) acell[i] = __ldg(g.acell32 + i);
  __syncthreads();

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  Rec32 &R = recs[warp];
  const int per_tile = MODE == MODE_MC ? 16 : 32;
  const int nc = MODE == MODE_MC ? g.nf : ncol;  // columns per point
  const int cbase = MODE == MODE_MC ? 0 : col0;
  const long long ntiles = (n + per_tile - 1) / per_tile;
  const long long nwarps = (long long)gridDim.x * kWarps;
  const unsigned lt = (1u << lane) - 1u;

  for (long long tile = (long long)blockIdx.x * kWarps + warp; tile < ntiles; tile += nwarps) {
    const long long e0 = tile * per_tile;
    const int ne = (int)(n - e0 < per_tile ? n - e0 : per_tile);

    // ---- phase 1: lane = point ----
    bool present;
    float x = 0.f, q2 = 0.f;
    long long ob;
    if (MODE == MODE_POINTS) {
      present = lane < ne;
      if (present) { x = xa[e0 + lane]; q2 = qa[e0 + lane]; }
      ob = (e0 + lane) * (long long)nc;
    } else {  // events: x1 = xa, x2 = xb
      const int e = lane >> 1;
      present = e < ne;
      if (present) {
        float x1 = xa[e0 + e], x2 = xb[e0 + e];
        q2 = x1 * x2 * s;
        x = (lane & 1) ? x2 : x1;
      }
      ob = (e0 + e) * (long long)(2 * g.nf + 1) + (lane & 1) * g.nf;
    }
    PointSites<float> ps;
    ps.cls = -1;
    if (present) ps = sites(g, xkeys, qkeys, xcell, qcell, rowqc, x, q2);
    unsigned inv = __ballot_sync(0xffffffffu, ps.cls == C_INVALID);
    if (lane == 0 && inv) atomicAdd(g.invalid, (unsigned long long)__popc(inv));
    if (MODE == MODE_MC && present && (lane & 1) == 0) out[ob + 2 * g.nf] = alphas_eval(g, akeys, acell, q2);
    if (MODE == MODE_POINTS && present && as_out) as_out[e0 + lane] = alphas_eval(g, akeys, acell, q2);
    // order the points by class (counting sort over the warp); in-grid points first
    int slot = 0, base = 0, nin = 0;
#pragma unroll
    for (int c = 0; c < NCLASS; c++) {
      const unsigned m = __ballot_sync(0xffffffffu, ps.cls == c);
      if (ps.cls == c) slot = base + __popc(m & lt);
      base += __popc(m);
      if (c == C_IN) nin = base;
    }
    const int np = base;
    if (present) store_point32(R, slot, ps, ob, g);
    __syncwarp();

    // ---- phase 2: items (point, column) ----
    const int dp = 32 / nc, dc = 32 - dp * nc;
    int p = lane / nc, c = lane - (lane / nc) * nc;
    for (int k = lane; k < np * nc; k += 32) {
      out[R.ob[p] + c] = p < nin ? eval_in32(g, R, p, cbase + c) : eval_item32(g, R, p, cbase + c);
      c += dc;
      p += dp;
      if (c >= nc) { c -= nc; p++; }
    }
    __syncwarp();
  }
}

// SQ: the input is Q, squared here (Q <= 0 or NaN is invalid; a square that
// overflows to infinity is invalid like Q^2 = inf).
template <typename T, bool SQ>
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
    if (SQ) q2 = q2 > T(0) ? q2 * q2 : T(-1);
    bool bad = present && !((q2 > T(0)) && (q2 < T(INFINITY)));
    unsigned inv = __ballot_sync(0xffffffffu, bad);
    if ((threadIdx.x & 31) == 0 && inv) atomicAdd(g.invalid, (unsigned long long)__popc(inv));
    if (present) {
      // FP64: the node position as the evaluation kernels take it (float-float
      // from the knots' exponents and significands, or the FP64 logarithm)
      if constexpr (sizeof(T) == 8)
        out[i] = g.ffpos ? alphas_ff(g, akeys, g.lnfff, g.lnfff2, q2, pos_tabs(g))
                         : alphas_eval(g, akeys, q2, bad ? 0.0 : tlog(q2, LogTabs{g.tlogtab, g.tloghtab}));
      else out[i] = alphas_eval(g, akeys, g.acell32, q2);
    }
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

static size_t xf32_smem(const GridView &g) { return smem32_layout(g).total; }

template <int MODE>
static int launch_xf32(const pdf_grid *grid, const float *xa, const float *qa, const float *xb, float s,
                       long long n, int col0, int ncol, float *out, cudaStream_t st, float *as_out = nullptr) {
  const GridView &g = grid->v;
  const size_t smem = xf32_smem(g);
  auto kern = k_xf32<MODE>;
  static LaunchCache cache;
  const int per_sm = cache.blocks_per_sm(kern, kThreads, smem);
  const int per_tile = MODE == MODE_MC ? 16 : 32;
  const long long ntiles = (n + per_tile - 1) / per_tile;
  long long blocks = (ntiles + kWarps - 1) / kWarps;
  const long long cap = (long long)num_sms() * per_sm;
  if (blocks > cap) blocks = cap;
  kern<<<(unsigned)blocks, kThreads, smem, st>>>(g, xa, qa, xb, s, n, col0, ncol, out, as_out);
  return check_launch(MODE == MODE_MC ? "pdf_mc_event kernel (FP32)" : "xfxq2 kernel (FP32)");
}

// One name for both precisions: FP32 here, FP64 in xf64.cu.
template <typename T, int MODE>
static int launch_xf(const pdf_grid *grid, const T *xa, const T *qa, const T *xb, T s, long long n, int col0,
                     int ncol, T *out, cudaStream_t st) {
  if constexpr (sizeof(T) == 8) return launch_xf64(grid, MODE, xa, qa, xb, s, n, col0, ncol, out, nullptr, st);
  else return launch_xf32<MODE>(grid, xa, qa, xb, s, n, col0, ncol, out, st);
}

template <typename T, bool SQ = false>
static int launch_alphas(const pdf_grid *grid, const T *q2, long long n, T *out, cudaStream_t st) {
  const GridView &g = grid->v;
  using K = typename std::conditional<sizeof(T) == 8, long long, int>::type;
  size_t smem = keys_bytes(g.na, sizeof(K));
  long long blocks = (n + kThreads - 1) / kThreads;
  long long cap = (long long)num_sms() * 8;
  if (blocks > cap) blocks = cap;
  k_alphas<T, SQ><<<(unsigned)blocks, kThreads, smem, st>>>(g, q2, n, out);
  return check_launch(SQ ? "alphas_q kernel" : "alphas_q2 kernel");
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

template <typename T, bool SQ = false>
static int do_alphas(const pdf_grid *g, const T *q, size_t n, T *out, cudaStream_t st) {
  const char *what = SQ ? "alphas_q" : "alphas_q2";
  int rc = check_common(g, q, q, out, n, what);
  if (rc) return rc;
  if (g->v.na == 0) return set_error(PDF_ERR_NO_ALPHAS, "%s: grid has no alpha_s nodes", what);
  if (n == 0) return PDF_OK;
  return launch_alphas<T, SQ>(g, q, (long long)n, out, st);
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
  // one member: the layout [1][n][nf] is the points layout, and the points
  // kernel gives the bits xfxq2_all_flavours gives
  if (g->v.nmem == 1) return launch_xf64(g, MODE_POINTS, x, q2, nullptr, 0.0, n, 0, g->v.nf, out, nullptr, st);
  return launch_xf64(g, MODE_MEMBERS, x, q2, nullptr, 0.0, n, 0, g->v.nf, out, nullptr, st);
}

// All flavours, and alpha_s into as_out when not null, in one pass.
int launch_all_f64(const pdf_grid *g, const double *x, const double *q2, long long n, double *out,
                   double *as_out, cudaStream_t st) {
  return launch_xf64(g, MODE_POINTS, x, q2, nullptr, 0.0, n, 0, g->v.nf, out, as_out, st);
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
extern "C" int xfxq2_all_flavours_alphas(const pdf_grid *g, const double *x, const double *q2, size_t n,
                                         double *out, double *alphas_out, cudaStream_t st) {
  int rc = check_common(g, x, q2, out, n, "xfxq2_all_flavours_alphas");
  if (rc) return rc;
  if (n > 0 && !alphas_out) return set_error(PDF_ERR_NULL, "xfxq2_all_flavours_alphas: alphas_out is NULL");
  if (g->v.na == 0) return set_error(PDF_ERR_NO_ALPHAS, "xfxq2_all_flavours_alphas: grid has no alpha_s nodes");
  if (n == 0) return PDF_OK;
  return launch_all_f64(g, x, q2, (long long)n, out, alphas_out, st);
}
extern "C" int xfxq2_all_flavours_alphas_f32(const pdf_grid *g, const float *x, const float *q2, size_t n,
                                             float *out, float *alphas_out, cudaStream_t st) {
  int rc = check_common(g, x, q2, out, n, "xfxq2_all_flavours_alphas_f32");
  if (rc) return rc;
  if (n > 0 && !alphas_out) return set_error(PDF_ERR_NULL, "xfxq2_all_flavours_alphas_f32: alphas_out is NULL");
  if (g->v.na == 0) return set_error(PDF_ERR_NO_ALPHAS, "xfxq2_all_flavours_alphas_f32: grid has no alpha_s nodes");
  if (n == 0) return PDF_OK;
  return launch_xf32<MODE_POINTS>(g, x, q2, nullptr, 0.f, (long long)n, 0, g->v.nf, out, st, alphas_out);
}
extern "C" int alphas_q2(const pdf_grid *g, const double *q2, size_t n, double *out, cudaStream_t st) {
  return do_alphas<double>(g, q2, n, out, st);
}
extern "C" int alphas_q2_f32(const pdf_grid *g, const float *q2, size_t n, float *out, cudaStream_t st) {
  return do_alphas<float>(g, q2, n, out, st);
}
extern "C" int alphas_q(const pdf_grid *g, const double *q, size_t n, double *out, cudaStream_t st) {
  return do_alphas<double, true>(g, q, n, out, st);
}
extern "C" int alphas_q_f32(const pdf_grid *g, const float *q, size_t n, float *out, cudaStream_t st) {
  return do_alphas<float, true>(g, q, n, out, st);
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
