// mc.cu -- pdf_mc_integrate: Monte Carlo integration driven by the PDF load
// of PDFFlow Sec. 4.1 (the VegasFlow use of Sec. 5).
//
// Per chunk of events, three launches on the caller's stream:
//   1. k_xf64<MODE_MC> generates the events (mc.cuh), writes each event's
//      s-hat = Q^2 = x1 x2 s, and for the events that pass the s-hat cut
//      all flavours at x1 and at x2 and alpha_s at Q^2 (an event below the
//      cut has weight zero whatever its PDFs: it is not evaluated, and when
//      no evaluated event can leave the grid the far launch is left out);
//   2. k_mc_weights turns each row into the event weight and reduces
//      (w, w^2, |w|) per block, in a fixed order;
//   3. k_mc_reduce adds the block sums, in a fixed order, to the running sums.
// The result is bit-reproducible for a given (seed, events, chunk).
#include <cmath>

#include "mc.cuh"
#include "pdf_internal.cuh"

namespace pdfgb {
namespace {

constexpr int kMcThreads = 256;
constexpr int kMcBlocks = 152 * 4;

struct McCols {
  int q[5], qb[5], g;  // columns of d, u, s, c, b, their antiquarks, the gluon
  int nf;
};

__device__ __forceinline__ double block_sum(double v, double *sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < kMcThreads / 32; w++) t += sh[w];
  return t;  // valid in thread 0
}

// Event weight (the toy leading-order observable of pdf_mc_integrate):
//   w = L^2 / s-hat * [sum_q e_q^2 (xf_q(x1) xf_qbar(x2) + xf_qbar(x1) xf_q(x2))
//                      + alpha_s^2 xf_g(x1) xf_g(x2)],  s-hat >= s-hat_min, else 0.
__global__ void __launch_bounds__(kMcThreads)
k_mc_weights(const double *__restrict__ ev, const double *__restrict__ shats, long long n, double shat_min,
             double lfac2, McCols c, double *__restrict__ part) {
  __shared__ double sh[kMcThreads / 32];
  const double e2[5] = {1.0 / 9.0, 4.0 / 9.0, 1.0 / 9.0, 4.0 / 9.0, 1.0 / 9.0};
  const int per = 2 * c.nf + 1;
  double sw = 0.0, sw2 = 0.0, sa = 0.0;
  for (long long i = (long long)blockIdx.x * kMcThreads + threadIdx.x; i < n; i += (long long)gridDim.x * kMcThreads) {
    const double shat = shats[i];  // x1 x2 s, as the event kernel took it
    double w = 0.0;
    if (shat >= shat_min) {
      const double *r1 = ev + i * per, *r2 = r1 + c.nf;
      double acc = 0.0;
#pragma unroll
      for (int k = 0; k < 5; k++) acc += e2[k] * (r1[c.q[k]] * r2[c.qb[k]] + r1[c.qb[k]] * r2[c.q[k]]);
      const double as = r1[2 * c.nf];
      acc += as * as * (r1[c.g] * r2[c.g]);
      w = lfac2 * acc / shat;
    }
    sw += w;
    sw2 += w * w;
    sa += fabs(w);
  }
  const double t0 = block_sum(sw, sh), t1 = block_sum(sw2, sh), t2 = block_sum(sa, sh);
  if (threadIdx.x == 0) {
    part[3 * blockIdx.x] = t0;
    part[3 * blockIdx.x + 1] = t1;
    part[3 * blockIdx.x + 2] = t2;
  }
}

__global__ void __launch_bounds__(kMcThreads) k_mc_reduce(const double *__restrict__ part, int nb, double *acc) {
  __shared__ double sh[kMcThreads / 32];
  for (int c = 0; c < 3; c++) {
    double v = 0.0;
    for (int b = threadIdx.x; b < nb; b += kMcThreads) v += part[3 * b + c];
    const double t = block_sum(v, sh);
    if (threadIdx.x == 0) acc[c] += t;
  }
}

int ensure_mc(pdf_grid *g, size_t cap) {
  if (g->mc_buf && g->mc_cap >= cap) return PDF_OK;
  if (g->mc_buf) { cudaFree(g->mc_buf); g->mc_buf = nullptr; }
  if (g->mc_part) { cudaFree(g->mc_part); g->mc_part = nullptr; }
  const size_t per = 2 * (size_t)g->v.nf + 1;  // a row per event, then the events' s-hat
  cudaError_t e = cudaMalloc(&g->mc_buf, cap * (per + 1) * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&g->mc_part, (3 * (size_t)kMcBlocks + 3) * sizeof(double));
  if (e != cudaSuccess) {
    if (g->mc_buf) cudaFree(g->mc_buf);
    g->mc_buf = nullptr;
    g->mc_part = nullptr;
    g->mc_cap = 0;
    return set_error(PDF_ERR_ALLOC, "pdf_mc_integrate: scratch for %zu events: %s", cap, cudaGetErrorString(e));
  }
  g->mc_acc = g->mc_part + 3 * kMcBlocks;
  g->mc_cap = cap;
  return PDF_OK;
}

}  // namespace
}  // namespace pdfgb

using namespace pdfgb;

extern "C" int pdf_mc_integrate(const pdf_grid *cg, const pdf_mc_config *cfg, unsigned long long first_event,
                                unsigned long long n_events, size_t chunk, double *sums, cudaStream_t st) {
  if (!cg || !cfg || !sums) return set_error(PDF_ERR_NULL, "pdf_mc_integrate: NULL argument");
  if (chunk < 1) return set_error(PDF_ERR_ARG, "pdf_mc_integrate: chunk must be >= 1");
  if (chunk > ((size_t)1 << 31)) return set_error(PDF_ERR_ARG, "pdf_mc_integrate: chunk %zu too large", chunk);
  const GridView &v = cg->v;
  if (v.na == 0) return set_error(PDF_ERR_NO_ALPHAS, "pdf_mc_integrate: grid has no alpha_s nodes");
  if (!(cfg->sqrt_s > 0.0) || !std::isfinite(cfg->sqrt_s))
    return set_error(PDF_ERR_ARG, "pdf_mc_integrate: sqrt_s must be positive and finite");
  if (!(cfg->x_min > 0.0) || !(cfg->x_min < v.xlast))
    return set_error(PDF_ERR_ARG, "pdf_mc_integrate: x_min must lie in (0, last x knot)");
  if (!(cfg->shat_min >= 0.0) || !std::isfinite(cfg->shat_min))
    return set_error(PDF_ERR_ARG, "pdf_mc_integrate: shat_min must be >= 0 and finite");
  McCols c{};
  c.nf = v.nf;
  for (int k = 0; k < 5; k++) {
    c.q[k] = pdf_grid_pid_column(cg, k + 1);
    c.qb[k] = pdf_grid_pid_column(cg, -(k + 1));
    if (c.q[k] < 0 || c.qb[k] < 0) return set_error(PDF_ERR_PID, "pdf_mc_integrate: the grid lacks pid +-%d", k + 1);
  }
  c.g = pdf_grid_pid_column(cg, 21);
  if (c.g < 0) return set_error(PDF_ERR_PID, "pdf_mc_integrate: the grid lacks the gluon (pid 21)");
  pdf_grid *g = const_cast<pdf_grid *>(cg);
  std::lock_guard<std::mutex> lock(g->mc_mu);  // one integration at a time per grid (shared scratch)
  const size_t cap = n_events < chunk ? (size_t)(n_events > 0 ? n_events : 1) : chunk;
  int rc = ensure_mc(g, cap);
  if (rc) return rc;

  const double s = cfg->sqrt_s * cfg->sqrt_s;
  McGen gen{};
  gen.seed = cfg->seed;
  gen.lxmin = log(cfg->x_min);
  gen.lxmax = log(v.xlast);
  gen.xmax = v.xlast;
  gen.on = 1;
  gen.et = v.texptab;
  // events that fail the s-hat cut get weight zero whatever their PDFs, and
  // k_mc_weights reads the rows of the others only: the event kernel skips
  // them (the same product x1 x2 s decides in both kernels)
  gen.cut = 1;
  gen.shat_min = cfg->shat_min;
  // With x in [x_min, x_max] (x_max capped, the lower end within a few ulp of
  // x_min) and Q^2 = x1 x2 s in [shat_min, fl(fl(x_max x_max) s)] (rounding is
  // monotonic) every evaluated event lies inside the grid when x_min clears
  // its first x knot and that Q^2 range lies in [Q2min, Q2max]: the far launch
  // would find nothing to do.
  gen.near_only = cfg->x_min * (1.0 - 1e-9) >= v.x0 && (v.xlast * v.xlast) * s <= v.q2max &&
                  cfg->shat_min >= v.q2min;
  // the event kernel leaves each event's s-hat after the rows: the weights
  // need no second generation of the events
  double *shats = g->mc_buf + cap * (2 * (size_t)v.nf + 1);
  gen.shat_out = shats;
  const double L = gen.lxmax - gen.lxmin;
  cudaError_t e = cudaMemsetAsync(g->mc_acc, 0, 3 * sizeof(double), st);
  for (unsigned long long off = 0; off < n_events && e == cudaSuccess && rc == PDF_OK; off += chunk) {
    const unsigned long long m = n_events - off < chunk ? n_events - off : chunk;
    gen.first = first_event + off;
    rc = launch_xf64(g, MODE_MC, nullptr, nullptr, nullptr, s, (long long)m, 0, 0, g->mc_buf, nullptr, st, &gen);
    if (rc) break;
    k_mc_weights<<<kMcBlocks, kMcThreads, 0, st>>>(g->mc_buf, shats, (long long)m, cfg->shat_min, L * L, c,
                                                    g->mc_part);
    k_mc_reduce<<<1, kMcThreads, 0, st>>>(g->mc_part, kMcBlocks, g->mc_acc);
    rc = check_launch("pdf_mc_integrate kernels");
  }
  if (rc) return rc;
  if (e == cudaSuccess) e = cudaMemcpyAsync(sums, g->mc_acc, 3 * sizeof(double), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return set_error(PDF_ERR_CUDA, "pdf_mc_integrate: %s", cudaGetErrorString(e));
  return PDF_OK;
}
