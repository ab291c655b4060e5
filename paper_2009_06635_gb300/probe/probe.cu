// probe.cu -- measurement and test hooks, linked into libpdfgb300_probe.so
// (not the evaluation library): an FMA-rate microbenchmark (the ALU ceiling
// of the FP64 and FP32 evaluation kernels; 8 independent chains per thread
// hide the FMA latency) and the evaluation kernels' elementary functions on
// given arguments.  It reads a grid handle's staged tables through the
// evaluation library's internal layout, so both libraries are built from the
// same headers.
#include <cstdarg>
#include <cstdio>

#include "pdf_gb300_probe.h"
#include "ffmath.cuh"
#include "ffpos.cuh"
#include "ffsplit.cuh"
#include "pdf_internal.cuh"

namespace {
thread_local char g_probe_err[256] = "";

int probe_error(int code, const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_probe_err, sizeof g_probe_err, fmt, ap);
  va_end(ap);
  return code;
}

int probe_launch(const char *what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return probe_error(PDF_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
  return PDF_OK;
}
}  // namespace

namespace pdfgb {

template <typename T>
__global__ void __launch_bounds__(256) k_fma(T a, T b, int iters, T *sink) {
  T c0 = (T)threadIdx.x, c1 = c0 + T(1), c2 = c0 + T(2), c3 = c0 + T(3);
  T c4 = c0 + T(4), c5 = c0 + T(5), c6 = c0 + T(6), c7 = c0 + T(7);
  for (int i = 0; i < iters; i++) {
    c0 = c0 * a + b; c1 = c1 * a + b; c2 = c2 * a + b; c3 = c3 * a + b;
    c4 = c4 * a + b; c5 = c5 * a + b; c6 = c6 * a + b; c7 = c7 * a + b;
  }
  T r = c0 + c1 + c2 + c3 + c4 + c5 + c6 + c7;
  if (r == T(-1.2345)) sink[threadIdx.x] = r;  // keeps the chains live
}

template <typename T>
static int probe(int iters, double *out) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  T *sink = nullptr;
  cudaEvent_t e0, e1;
  if (cudaMalloc(&sink, 256 * sizeof(T)) != cudaSuccess) return probe_error(PDF_ERR_ALLOC, "probe: cudaMalloc");
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int blocks = sms * 8;
  k_fma<T><<<blocks, 256>>>(T(0.999999), T(1e-7), iters / 8 + 1, sink);  // warm-up
  cudaEventRecord(e0);
  k_fma<T><<<blocks, 256>>>(T(0.999999), T(1e-7), iters, sink);
  cudaEventRecord(e1);
  cudaError_t e = cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(sink);
  if (e != cudaSuccess) return probe_error(PDF_ERR_CUDA, "probe: %s", cudaGetErrorString(e));
  *out = 2.0 * 8.0 * (double)iters * blocks * 256 / (ms * 1e-3);
  return probe_launch("probe");
}

// The evaluation kernels' own elementary functions, elementwise (tang.cuh,
// ffmath.cuh; the float-float ones take their argument rounded to a float pair).
__global__ void k_math(GridView g, int fn, const double *a, const double *b, long long n, double *out) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const FFTabs FT{g.fflog, g.ffexp};
  switch (fn) {
    case 0: out[i] = tlog(a[i], LogTabs{g.tlogtab, g.tloghtab}); break;
    case 1: out[i] = texp(a[i], g.texptab); break;
    case 2: out[i] = ddiv(a[i], b[i]); break;
    case 3: out[i] = ff_to_d(ff_log(ff_of(a[i]), FT)); break;
    case 4: out[i] = ff_to_d(ff_exp(ff_of(a[i]), FT)); break;
    case 5: out[i] = ff_to_d(ff_div(ff_of(a[i]), ff_of(b[i]))); break;
    case 8:  // the integer split of a (ffsplit.cuh): hi + lo, NaN outside its range
    case 9: {  // hi alone
      if (!ff_safe(a[i], 50)) {
        out[i] = NAN;
        break;
      }
      const ff2 v = ff_split50(a[i]);
      out[i] = fn == 8 ? ff_to_d(v) : f2d(v.h);
      break;
    }
    default: {  // 6, 7: t and 1 - t of x = a[i] in its x cell (ffpos.cuh), a[i] in [x0, x_last]
      const long long *xk = reinterpret_cast<const long long *>(g.xk);
      const long long kx = __double_as_longlong(a[i]);
      if (!(kx >= xk[0] && kx <= xk[g.nx - 1])) {  // outside the knots (or not a positive number)
        out[i] = NAN;
        break;
      }
      const int c = search_cell(xk, g.nx, g.xstep, kx);
      const bool k1 = kx != xk[c];
      ff2 t, ts;
      ff_cell_pos2(kx, xk[c], k1 ? xk[c + 1] : 0, g.xposff[c], k1 ? g.xposff[c + 1] : make_float4(0.f, 0.f, 0.f, 0.f),
                   g.lnfff, g.lnfff2, t, ts);
      out[i] = ff_to_d(fn == 6 ? t : ts);
      break;
    }
  }
}

}  // namespace pdfgb

extern "C" int pdf_probe_math(const pdf_grid *grid, int fn, const double *a, const double *b, size_t n,
                              double *out, cudaStream_t stream) {
  using namespace pdfgb;
  if (!grid || (n > 0 && (!a || !out || ((fn == 2 || fn == 5) && !b))))
    return probe_error(PDF_ERR_NULL, "pdf_probe_math: NULL argument");
  if (fn < 0 || fn > 9) return probe_error(PDF_ERR_ARG, "pdf_probe_math: fn must be 0 .. 9");
  if ((fn == 6 || fn == 7) && !grid->v.ffpos)
    return probe_error(PDF_ERR_ARG, "pdf_probe_math: the grid takes no float-float positions");
  if (n == 0) return PDF_OK;
  k_math<<<(unsigned)((n + 255) / 256), 256, 0, stream>>>(grid->v, fn, a, b, (long long)n, out);
  return probe_launch("pdf_probe_math");
}

extern "C" int pdf_probe_fma_rate(int precision, int iters, double *flops_per_s) {
  using namespace pdfgb;
  if (!flops_per_s) return probe_error(PDF_ERR_NULL, "pdf_probe_fma_rate: NULL output");
  if (iters < 1 || iters > (1 << 24)) return probe_error(PDF_ERR_ARG, "pdf_probe_fma_rate: iters out of range");
  if (precision == 64) return probe<double>(iters, flops_per_s);
  if (precision == 32) return probe<float>(iters, flops_per_s);
  return probe_error(PDF_ERR_ARG, "pdf_probe_fma_rate: precision must be 32 or 64");
}

extern "C" const char *pdf_probe_last_error(void) { return g_probe_err; }
