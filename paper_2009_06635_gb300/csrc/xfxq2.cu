// xfxq2.cu -- FP32 evaluation kernel for x f(x, Q^2), the alpha_s kernel,
// and the C entry points of both precisions (FP64 evaluation: xf64.cu).
//
// One warp owns a tile of 32 query points (16 events in the Monte Carlo
// layout).  Phase 1 (lane = point): read x and Q^2 (coalesced), classify
// against the grid edges, search the cells on the raw bit patterns (knots in
// shared memory), and record the Bernstein weights of the patch sites and the
// continuation parameters of the point.  Phase 2, per point (warp-uniform,
// so classes never diverge): in-grid points spread (column, row pair) over
// the lanes, one float4 pair of control points each and one shuffle per
// evaluation; continuation points use four lanes per item, each loading one
// float4 row of control points, reduced with two shuffles.  The FP32 path is
// bound by the L1/L2 gather, not arithmetic.
#include <cmath>
#include <type_traits>

#include "sites.cuh"

namespace pdfgb {

constexpr int kWarps = 8;
constexpr int kThreads = 32 * kWarps;

// Per-warp record of the points of one tile, indexed by class-sorted slot.
// W holds, per slot, Bx0 | Bx1 | Bq0 | Bq1.
template <typename T>
struct WarpRec {
  int cls[32], orig[32], xc0[32], xc1[32], qc0[32], qc1[32];
  int off4[32];  // FP32 in-grid points: float4 offset of the cell's first flavour block
  T W[16][33];  // padded: rows of one slot fall in different banks
  T px[32], pq[32], lr[32], as[32];
};

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
__device__ __forceinline__ void store_weights(WarpRec<float> &R, int slot, const PointSites<float> &ps) {
  float bx0[4], bx1[4], bq0[4], bq1[4];
  bernstein<float>(ps.t0, ps.ts0, bx0);
  bernstein<float>(ps.t1, 1.f - ps.t1, bx1);
  bernstein<float>(ps.u0, ps.us0, bq0);
  bernstein<float>(ps.u1, 1.f - ps.u1, bq1);
#pragma unroll
  for (int k = 0; k < 4; k++) {
    R.W[k][slot] = bx0[k];
    R.W[4 + k][slot] = bx1[k];
    R.W[8 + k][slot] = bq0[k];
    R.W[12 + k][slot] = bq1[k];
  }
}

// MODE_POINTS: points xa[n], qa[n]; out[n][ncol] for columns col0..col0+ncol-1.
// MODE_MC:     events xa[n] (x1), xb[n] (x2), Q^2 = x1 x2 s; out[n][2 nf + 1].
template <int MODE>
__global__ void __launch_bounds__(kThreads, 4)
k_xf32(GridView g, const float *__restrict__ xa, const float *__restrict__ qa, const float *__restrict__ xb,
       float s, long long n, int col0, int ncol, float *__restrict__ out) {
  extern __shared__ __align__(16) unsigned char smem[];
  int *xkeys = reinterpret_cast<int *>(smem);
  int *qkeys = reinterpret_cast<int *>(smem + keys_bytes(g.nx, 4));
  int *akeys = reinterpret_cast<int *>(smem + keys_bytes(g.nx, 4) + keys_bytes(g.nrows, 4));
  size_t rec_off = keys_bytes(g.nx, 4) + keys_bytes(g.nrows, 4) + (MODE == MODE_MC ? keys_bytes(g.na, 4) : 0);
  WarpRec<float> *recs = reinterpret_cast<WarpRec<float> *>(smem + rec_off);
  load_keys<float>(g, xkeys, 0);
  load_keys<float>(g, qkeys, 1);
  if (MODE == MODE_MC) load_keys<float>(g, akeys, 2);
  __syncthreads();

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  WarpRec<float> &R = recs[warp];
  const int per_tile = MODE == MODE_MC ? 16 : 32;
  const int per = MODE == MODE_MC ? 2 * g.nf + 1 : ncol;  // outputs per tile unit
  const int r = lane & 3;                                  // row of a four-lane item
  const unsigned gm = 0xFu << (lane & ~3);
  const long long ntiles = (n + per_tile - 1) / per_tile;
  const long long nwarps = (long long)gridDim.x * kWarps;

  for (long long tile = (long long)blockIdx.x * kWarps + warp; tile < ntiles; tile += nwarps) {
    const long long e0 = tile * per_tile;
    const int ne = (int)(n - e0 < per_tile ? n - e0 : per_tile);

    // ---- phase 1: lane = point ----
    bool present;
    float x = 0.f, q2 = 0.f;
    if (MODE == MODE_POINTS) {
      present = lane < ne;
      if (present) { x = xa[e0 + lane]; q2 = qa[e0 + lane]; }
    } else {  // events: x1 = xa, x2 = xb
      const int e = lane >> 1;
      present = e < ne;
      if (present) {
        float x1 = xa[e0 + e], x2 = xb[e0 + e];
        q2 = x1 * x2 * s;
        x = (lane & 1) ? x2 : x1;
      }
    }
    PointSites<float> ps;
    ps.cls = NCLASS;
    if (present) ps = sites(g, xkeys, qkeys, x, q2);
    unsigned inv = __ballot_sync(0xffffffffu, present && ps.cls == C_INVALID);
    if (lane == 0 && inv) atomicAdd(g.invalid, (unsigned long long)__popc(inv));

    const int slot = lane;  // phase 2 walks the points in order: no sort needed
    R.cls[slot] = ps.cls; R.orig[slot] = lane;
    R.off4[slot] = ((ps.qc0 * g.nx + ps.xc0) * g.nf + col0) * 4;
    R.xc0[slot] = ps.xc0; R.xc1[slot] = ps.xc1; R.qc0[slot] = ps.qc0; R.qc1[slot] = ps.qc1;
    R.px[slot] = ps.px; R.pq[slot] = ps.pq; R.lr[slot] = ps.lr;
    if (present && ps.cls != C_INVALID) store_weights(R, slot, ps);
    if (MODE == MODE_MC && (lane & 1) == 0) R.as[lane >> 1] = present ? alphas_eval(g, akeys, q2) : 0.f;
    __syncwarp();

    // ---- phase 2: per point, lanes over (column, row) ----
    if (MODE == MODE_POINTS && ncol == 1) {  // one column: a lane per point
      if (lane < ne) out[e0 + R.orig[lane]] = eval_point32(g, R, lane, col0);
    } else {
      const int nc = MODE == MODE_MC ? g.nf : ncol;
      const int npts = MODE == MODE_MC ? 2 * ne : ne;
      for (int q = 0; q < npts; q++) {  // warp-uniform: no divergence by class
        const long long ob = MODE == MODE_POINTS ? (e0 + R.orig[q]) * (long long)ncol
                                                 : (e0 + (q >> 1)) * (long long)per + (q & 1) * g.nf;
        if (R.cls[q] == C_IN) {
          // the point's column blocks are contiguous: lane k owns rows 2h, 2h+1
          // (h = k & 1) of column k >> 1, 32 bytes at cell_base + 8 k floats
          const float4 *cbp = reinterpret_cast<const float4 *>(g.coef32) + R.off4[q];
          const float b0 = R.W[0][q], b1 = R.W[1][q], b2 = R.W[2][q], b3 = R.W[3][q];
          const int hr = lane & 1;
          const float bqa = R.W[8 + 2 * hr][q], bqb = R.W[9 + 2 * hr][q];
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
            const float v = eval_item32(g, R, q, col0 + f, r, gm);
            if (r == 0) out[ob + f] = v;
          }
        }
      }
      if (MODE == MODE_MC && lane < ne) out[(e0 + lane) * (long long)per + 2 * g.nf] = R.as[lane];
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
    if (present) {
      if constexpr (sizeof(T) == 8) out[i] = alphas_eval(g, akeys, q2, bad ? 0.0 : tlog(q2, g.tlogtab));
      else out[i] = alphas_eval(g, akeys, q2);
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

template <int MODE>
static size_t xf32_smem(const GridView &g) {
  return keys_bytes(g.nx, 4) + keys_bytes(g.nrows, 4) + (MODE == MODE_MC ? keys_bytes(g.na, 4) : 0) +
         kWarps * sizeof(WarpRec<float>);
}

template <int MODE>
static int launch_xf32(const pdf_grid *grid, const float *xa, const float *qa, const float *xb, float s,
                       long long n, int col0, int ncol, float *out, cudaStream_t st) {
  const GridView &g = grid->v;
  const size_t smem = xf32_smem<MODE>(g);
  auto kern = k_xf32<MODE>;
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem);
  if (per_sm < 1) per_sm = 1;
  const int per_tile = MODE == MODE_MC ? 16 : 32;
  const long long ntiles = (n + per_tile - 1) / per_tile;
  long long blocks = (ntiles + kWarps - 1) / kWarps;
  const long long cap = (long long)num_sms() * per_sm;
  if (blocks > cap) blocks = cap;
  kern<<<(unsigned)blocks, kThreads, smem, st>>>(g, xa, qa, xb, s, n, col0, ncol, out);
  return check_launch(MODE == MODE_MC ? "pdf_mc_event kernel (FP32)" : "xfxq2 kernel (FP32)");
}

// One name for both precisions: FP32 here, FP64 in xf64.cu.
template <typename T, int MODE>
static int launch_xf(const pdf_grid *grid, const T *xa, const T *qa, const T *xb, T s, long long n, int col0,
                     int ncol, T *out, cudaStream_t st) {
  if constexpr (sizeof(T) == 8) return launch_xf64(grid, MODE, xa, qa, xb, s, n, col0, ncol, out, nullptr, st);
  else return launch_xf32<MODE>(grid, xa, qa, xb, s, n, col0, ncol, out, st);
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
  return launch_xf64(g, MODE_MEMBERS, x, q2, nullptr, 0.0, n, 0, g->v.nf, out, nullptr, st);
}

// Used by the host-memory path.
int launch_alphas_f64(const pdf_grid *g, const double *q2, long long n, double *out, cudaStream_t st) {
  return launch_alphas<double>(g, q2, n, out, st);
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
