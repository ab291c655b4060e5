// noalloc.cu -- a host-buffer evaluation entry point that allocates nothing.
//
// xfxq2_all_flavours_host stages its batches through device buffers that the
// grid allocates with cudaMalloc on first use.  Some callers cannot let a
// library do that: an event generator or integrator that calls the PDF from
// inside its own tight loop, where a cudaMalloc/cudaFree would synchronise
// the whole device and stall the pipeline; a host program whose device memory
// is entirely owned by another pool or framework, where an allocation behind
// its back can fail or fragment the pool; a process that must reach a steady
// state with no allocation at all after start-up.  For them,
// xfxq2_all_flavours_host_noalloc stages through a fixed array compiled into
// the library instead.
//
// The array is a file-scope __device__ symbol of kScratchDoubles doubles
// (16 MiB); every GPU on which the library's kernels are loaded holds it for
// the life of the process.  Host code cannot use the symbol's name as a
// device address, so the first call on each device looks the address up with
// cudaGetSymbolAddress (with that device current) and caches it.
#include <mutex>

#include "pdf_internal.cuh"

using namespace pdfgb;

namespace {

constexpr size_t kScratchDoubles = (size_t)1 << 21;  // 16 MiB
static __device__ __align__(256) double g_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_lock;
double *g_scratch_addr[kMaxDevices] = {};

// Device address of g_scratch on the current device (looked up once).
int scratch_address(double **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return set_error(PDF_ERR_CUDA, "no-alloc path: cudaGetDevice: %s", cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return set_error(PDF_ERR_ARG, "no-alloc path: device %d out of range", dev);
  std::lock_guard<std::mutex> hold(g_lock);
  if (!g_scratch_addr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess || !p)
      return set_error(PDF_ERR_CUDA, "no-alloc path: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
    g_scratch_addr[dev] = static_cast<double *>(p);
  }
  *out = g_scratch_addr[dev];
  return PDF_OK;
}

// Largest batch the array holds: x, Q^2, alpha_s and nflav outputs per point.
size_t max_points(const pdf_grid *g) { return kScratchDoubles / (3 + (size_t)g->v.nf); }

}  // namespace

extern "C" int xfxq2_all_flavours_host_noalloc(const pdf_grid *g, const double *x, const double *q2, size_t n,
                                               double *out, double *alphas_out, cudaStream_t stream) {
  if (!g) return set_error(PDF_ERR_NULL, "xfxq2_all_flavours_host_noalloc: grid is NULL");
  if (n > 0 && (!x || !q2 || !out))
    return set_error(PDF_ERR_NULL, "xfxq2_all_flavours_host_noalloc: NULL array");
  if (alphas_out && g->v.na == 0)
    return set_error(PDF_ERR_NO_ALPHAS, "xfxq2_all_flavours_host_noalloc: grid has no alpha_s nodes");
  const size_t cap = max_points(g);
  if (n > cap)
    return set_error(PDF_ERR_ARG,
                     "xfxq2_all_flavours_host_noalloc: n = %zu exceeds the fixed scratch capacity of %zu points "
                     "for %d flavours (2^21 doubles hold x, Q^2, alpha_s and nflav outputs per point)",
                     n, cap, g->v.nf);
  if (n == 0) return PDF_OK;
  double *base = nullptr;
  int rc = scratch_address(&base);
  if (rc) return rc;
  // layout: x [n] | Q^2 [n] | alpha_s [n] | xf [n][nflav]; every word read is
  // written first by this call, so nothing needs clearing.
  double *sx = base, *sq = base + n, *sa = base + 2 * n, *so = base + 3 * n;
  const int nf = g->v.nf;
  cudaError_t e = cudaMemcpyAsync(sx, x, n * sizeof(double), cudaMemcpyHostToDevice, stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(sq, q2, n * sizeof(double), cudaMemcpyHostToDevice, stream);
  if (e != cudaSuccess)
    return set_error(PDF_ERR_CUDA, "xfxq2_all_flavours_host_noalloc: copy in: %s", cudaGetErrorString(e));
  // all flavours and alpha_s in one pass (ln Q^2 taken once; the same bits
  // as the two separate kernels)
  rc = launch_all_f64(g, sx, sq, (long long)n, so, alphas_out ? sa : nullptr, stream);
  if (rc) return rc;
  e = cudaMemcpyAsync(out, so, n * nf * sizeof(double), cudaMemcpyDeviceToHost, stream);
  if (e == cudaSuccess && alphas_out)
    e = cudaMemcpyAsync(alphas_out, sa, n * sizeof(double), cudaMemcpyDeviceToHost, stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess)
    return set_error(PDF_ERR_CUDA, "xfxq2_all_flavours_host_noalloc: %s", cudaGetErrorString(e));
  return PDF_OK;
}
