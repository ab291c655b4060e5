// host_io.cu -- xfxq2_all_flavours_host: host buffers in, host buffers out.
//
// The batch is cut into chunks that rotate over three streams the grid owns; each chunk is copied in, evaluated and copied out on its stream, so
// the copy-in of one chunk, the kernel of another and the copy-out of a third
// overlap (the copy engines and the SMs work at the same time).  The output
// (8 nf bytes per point against 16 in) sets the pace: the device-to-host
// link is busy from the first copy-out to the end, so the first chunks are
// small (1/8, 1/4, 1/2 of a full one) to start that copy-out early.  With pinned
// host memory the copies are asynchronous DMA; with pageable memory they are
// correct but serialise.  The device staging buffers belong to the grid and
// are reused across calls.
#include "pdf_internal.cuh"

using namespace pdfgb;

static const size_t kChunk = (size_t)1 << 20;  // points per chunk

static int ensure_io(pdf_grid *g) {
  if (g->io_buf[0]) return PDF_OK;
  const size_t bytes = kChunk * (3 + (size_t)g->v.nf) * sizeof(double);
  for (int k = 0; k < pdf_grid::kIoStreams; k++) {
    cudaError_t e = cudaStreamCreateWithFlags(&g->io_stream[k], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMalloc(&g->io_buf[k], bytes);
    if (e != cudaSuccess) {
      for (int j = 0; j <= k; j++) {
        if (g->io_buf[j]) { cudaFree(g->io_buf[j]); g->io_buf[j] = nullptr; }
        if (g->io_stream[j]) { cudaStreamDestroy(g->io_stream[j]); g->io_stream[j] = nullptr; }
      }
      return set_error(PDF_ERR_ALLOC, "xfxq2_all_flavours_host: staging buffers: %s", cudaGetErrorString(e));
    }
  }
  g->io_cap = kChunk;
  return PDF_OK;
}

extern "C" int xfxq2_all_flavours_host(const pdf_grid *cg, const double *x, const double *q2, size_t n,
                                       double *out, double *alphas_out) {
  if (!cg) return set_error(PDF_ERR_NULL, "xfxq2_all_flavours_host: grid is NULL");
  if (n > 0 && (!x || !q2 || !out)) return set_error(PDF_ERR_NULL, "xfxq2_all_flavours_host: NULL array");
  if (alphas_out && cg->v.na == 0)
    return set_error(PDF_ERR_NO_ALPHAS, "xfxq2_all_flavours_host: grid has no alpha_s nodes");
  if (n == 0) return PDF_OK;
  pdf_grid *g = const_cast<pdf_grid *>(cg);
  std::lock_guard<std::mutex> lock(g->io_mu);  // one host-buffer call at a time per grid
  int rc = ensure_io(g);
  if (rc) return rc;
  const int nf = g->v.nf;
  cudaError_t e = cudaSuccess;
  size_t c = 0, m = 0;
  for (size_t off = 0; off < n && e == cudaSuccess && rc == PDF_OK; off += m, c++) {
    const size_t want = c < 3 ? g->io_cap >> (3 - c) : g->io_cap;  // ramp: 1/8, 1/4, 1/2, then whole chunks
    m = n - off < want ? n - off : want;
    const int k = (int)(c % pdf_grid::kIoStreams);
    cudaStream_t st = g->io_stream[k];
    double *dx = static_cast<double *>(g->io_buf[k]);
    double *dq = dx + g->io_cap;
    double *da = dq + g->io_cap;
    double *dout = da + g->io_cap;
    e = cudaMemcpyAsync(dx, x + off, m * sizeof(double), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dq, q2 + off, m * sizeof(double), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) rc = launch_all_f64(g, dx, dq, (long long)m, dout, alphas_out ? da : nullptr, st);
    if (e == cudaSuccess && rc == PDF_OK)
      e = cudaMemcpyAsync(out + off * nf, dout, m * nf * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && rc == PDF_OK && alphas_out)
      e = cudaMemcpyAsync(alphas_out + off, da, m * sizeof(double), cudaMemcpyDeviceToHost, st);
  }
  for (int k = 0; k < pdf_grid::kIoStreams; k++) {
    const cudaError_t ek = cudaStreamSynchronize(g->io_stream[k]);
    if (e == cudaSuccess) e = ek;
  }
  if (rc) return rc;
  if (e != cudaSuccess) return set_error(PDF_ERR_CUDA, "xfxq2_all_flavours_host: %s", cudaGetErrorString(e));
  return PDF_OK;
}
