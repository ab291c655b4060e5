/*
 * pdf_gb300_probe.h -- measurement and test hooks, built as a library of
 * their own (libpdfgb300_probe.so) beside the evaluation library; not part
 * of its C ABI, and the paper has no counterpart.
 *
 * pdf_probe_fma_rate measures the arithmetic ceilings that bound the
 * evaluation kernels, so a benchmark can state roofline fractions against
 * numbers taken on the same GPU; pdf_probe_math runs the kernels' own
 * elementary functions on given arguments, for tests against the C library.
 * Errors are reported by return code and pdf_probe_last_error().
 */
#ifndef PDF_GB300_PROBE_H
#define PDF_GB300_PROBE_H

#include "pdf_gb300.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Sustained fused-multiply-add rate of the current device: every thread of a
 * grid of (SMs x 8) blocks of 256 threads runs 8 independent FMA chains of
 * `iters` steps in registers.  precision: 64 (DFMA) or 32 (FFMA).
 * *flops_per_s receives 2 x FMAs / elapsed seconds (CUDA events).
 * Synchronous; returns PDF_OK or a PDF_ERR_* code. */
PDF_API int pdf_probe_fma_rate(int precision, int iters, double *flops_per_s);

/* The evaluation kernels' own elementary functions, elementwise on n DEVICE
 * values, for testing them against the C library: fn 0: out = ln a
 * (table-driven, Tang's method; within 2 ulp or 2e-17 absolute); fn 1:
 * out = e^a (within 2 ulp); fn 2: out = a / b (reciprocal approximation and
 * Newton steps, within 2 ulp); fn 3, 4, 5: the float-float logarithm,
 * exponential and quotient of the continuation rules, on a (and b) rounded to
 * float pairs (ln a within 2e-14 + 2e-14 |ln a| absolute for a in [2^-100, 2^100];
 * e^a within (1 + |a|) 1e-14 relative for |a| < 64; a / b within 4e-14
 * relative); fn 6, 7: the position t of x = a in its x cell and 1 - t, as
 * the evaluation kernels take it in float-float (ffpos.cuh; NaN for a
 * outside [x0, x_last]; PDF_ERR_ARG on a grid that keeps the FP64
 * positions); fn 8, 9: the adjoint's split of a double into a float pair on
 * the integer pipe (ffsplit.cuh), hi + lo and hi alone (hi the top 24
 * significant bits of a, hi + lo within 2^-48 |a|; NaN for a outside 0 and
 * 2^-50 <= |a| < 2^50).  b may be NULL unless fn is 2 or 5.  The tables are the
 * grid's (a handle of the evaluation library, loaded in the same process).
 * Asynchronous on `stream`. */
PDF_API int pdf_probe_math(const pdf_grid *grid, int fn, const double *a, const double *b, size_t n,
                           double *out, cudaStream_t stream);

/* Description of the last probe error on the calling thread ("" if none). */
PDF_API const char *pdf_probe_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* PDF_GB300_PROBE_H */
