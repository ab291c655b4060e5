/*
 * pdf_surrogate.h -- learned surrogate of the PDF interpolator.
 *
 * No counterpart in the paper: a growth axis that replaces the
 * interpolation of PDFFlow Sec. 2.2 by a small network where the network is
 * accurate enough, with the interpolator as fallback and as the reference
 * for the network's error.
 *
 * Network: (ln x, ln Q^2) scaled to [-1, 1]^2 -> 32 Fourier features
 * (sin and cos of pi (F z), F a fixed [16][2] matrix) -> four layers of width
 * 128 with SiLU -> one output per flavour y_f, mapped to xf_f by the
 * surrogate's target:
 *   PDF_SURR_ASINH     xf_f = c_f sinh(y_f), trained on asinh(xf_f / c_f),
 *                      c_f = 1e-5 max |xf_f| over the grid's knots (a signed
 *                      logarithm: steep where xf_f changes sign);
 *   PDF_SURR_ENVELOPE  xf_f = E_f(x) y_f, trained on xf_f / E_f(x), with
 *                      E_f(x_i) = max over the Q knots of |xf_f(x_i, Q)| (at
 *                      least c_f), ln E_f linear in ln x between x knots and
 *                      tabulated at 1025 equal steps of ln x over the grid
 *                      (the network then learns an O(1) function, smooth
 *                      through the zeros of xf_f);
 *   PDF_SURR_RESIDUAL  xf_f = B_f + 2^-10 E_f(x) y_f, trained on
 *                      (xf_f - B_f) / (2^-10 E_f(x)) clipped to [-32, 32]
 *                      (where the base misses by more than 3% of E_f the
 *                      cell fails the error map anyway): the network corrects a
 *                      base B_f, bilinear in the scaled coordinates on a
 *                      uniform 257 x 257 table of the FP64 interpolator (FP32,
 *                      built when the surrogate is made), whose own error is
 *                      ~1e-3 of E_f; the network's BF16 error then acts on a
 *                      term of that size.  The inference kernel forms B_f
 *                      from its four table nodes in its epilogue.
 * Products run on the BF16 tensor cores (tcgen05) with FP32 accumulation;
 * BF16 weight copies are made from FP32 master weights.
 * The parameter vector is flat FP32: W1 [128][32], b1 [128], W2..W4
 * [128][128], b2..b4 [128], W5 [nflav][128], b5 [nflav] (W as [out][in]).
 *
 * All array arguments are DEVICE memory unless noted; calls return PDF_OK or
 * a PDF_ERR_* code (see pdf_gb300.h).  At most 16 flavours.  The calls that
 * use the surrogate's own buffers (training, loss/gradient, error map,
 * evaluation with fallback, setting parameters) are serialised per
 * surrogate; pdf_surrogate_eval uses none and runs concurrently.  A grid
 * passed to training, the error map or the fallback must have as many
 * flavours as the surrogate's own (PDF_ERR_ARG otherwise).
 */
#ifndef PDF_SURROGATE_H
#define PDF_SURROGATE_H

#include "pdf_gb300.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pdf_surrogate pdf_surrogate;

typedef struct {
  int batch;                /* points per step                                   */
  int steps;                /* optimiser steps                                   */
  float lr, lr_min;         /* Adam learning rate: linear warm-up, cosine decay  */
  int warmup;               /* warm-up steps                                     */
} pdf_train_config;

#define PDF_SURR_ASINH 0
#define PDF_SURR_ENVELOPE 1
#define PDF_SURR_RESIDUAL 2

/* Make a surrogate for `grid` from HOST parameters (flat FP32, see above)
 * and HOST frequencies freq[16][2]; scratch for batches of up to max_batch
 * points is allocated here.  pdf_surrogate_create uses PDF_SURR_ASINH;
 * _ex takes the target (PDF_ERR_ARG if unknown).  Synchronous. */
PDF_API int pdf_surrogate_create(const pdf_grid *grid, const float *params, const float *freq, int max_batch,
                                 pdf_surrogate **out);
PDF_API int pdf_surrogate_create_ex(const pdf_grid *grid, const float *params, const float *freq, int max_batch,
                                    int target, pdf_surrogate **out);
PDF_API int pdf_surrogate_free(pdf_surrogate *s);
PDF_API int pdf_surrogate_nparams(const pdf_surrogate *s, size_t *n);
/* Copy the FP32 master parameters to / from HOST memory (synchronous). */
PDF_API int pdf_surrogate_get_params(const pdf_surrogate *s, float *params);
PDF_API int pdf_surrogate_set_params(pdf_surrogate *s, const float *params);

/* One forward and backward pass on n <= max_batch points with given target
 * values xf [n][nflav] (FP64): *loss (HOST) is the mean-square error of the
 * targets (asinh or envelope-scaled, by the surrogate's target), grad (HOST,
 * nparams FP32) its gradient.  Synchronous. */
PDF_API int pdf_surrogate_loss_grad(pdf_surrogate *s, const double *x, const double *q2, const double *xf,
                                    size_t n, double *loss, float *grad);

/* The intermediate values of the last pdf_surrogate_loss_grad pass, for
 * checking each stage of the GPU computation on its own inputs: out (HOST,
 * FP32) receives [n][cols] of
 *   what 0: the bfloat16 activations h_layer (layer 0: the 32 features; 1..4
 *           the SiLU outputs, 128 columns), as stored;
 *   what 1: the FP32 pre-activations z_layer of the SiLU layers (0..3, 128);
 *   what 2: the bfloat16 backward signals of layer `layer` (0..3: 128
 *           columns, dL/dz; 4: the 16 padded output columns, dL/dy);
 *   what 3: the FP32 outputs y (layer 0; 16 padded columns);
 *   what 4: the FP32 targets (layer 0; 16 padded columns).
 * PDF_ERR_ARG before any such pass or for another (what, layer).  Synchronous. */
PDF_API int pdf_surrogate_trace(pdf_surrogate *s, int what, int layer, float *out);

/* Train on the n points (x, q2), targets from the FP64 interpolator of
 * `grid`, batches taken in order.  *final_loss (HOST, may be NULL) is the
 * last batch's loss.  Enqueued on `stream`; returns after the last step. */
PDF_API int pdf_surrogate_train(pdf_surrogate *s, const pdf_grid *grid, const double *x, const double *q2,
                                size_t n, const pdf_train_config *cfg, double *final_loss, cudaStream_t stream);

/* Network output for n points inside the grid: out [n][nflav] FP32.
 * Inference runs on the tensor cores with bounded waits; a wait that runs
 * out (never expected) is reported by the next pdf_surrogate_build_error_map
 * or pdf_surrogate_eval_fallback as PDF_ERR_CUDA. */
PDF_API int pdf_surrogate_eval(const pdf_surrogate *s, const double *x, const double *q2, size_t n, float *out,
                               cudaStream_t stream);

/* Error map: evaluate the network and the FP64 interpolator on n validation
 * points, record per tile of a 64 x 64 partition of the scaled (ln x, ln Q^2)
 * square the largest error |s - v| / max(|v|, c_f) over points and
 * flavours, and accept a tile when it was sampled and its error is at most
 * `threshold`.  With PDF_SURR_RESIDUAL the base alone (the network's term
 * left out) is measured on the same points too, and a tile is served by the
 * more accurate of the two among those within the threshold.  stats (HOST,
 * may be NULL) receives [tiles accepted, tiles sampled, largest error,
 * median tile error], a tile's error being that of the way it is served (of
 * the better way where neither passes).  Synchronous. */
PDF_API int pdf_surrogate_build_error_map(pdf_surrogate *s, const pdf_grid *grid, const double *x,
                                          const double *q2, size_t n, double threshold, double *stats);

/* The last error map's tile states into HOST states[64 * 64], tile (tx, tq)
 * at tq * 64 + tx, tx = floor((z0 + 1) 32), tq = floor((z1 + 1) 32) of the
 * scaled coordinates (FP32): 0 the interpolator, 1 the network, 2 the
 * residual target's base alone.  PDF_ERR_ARG before any error map.
 * Synchronous. */
PDF_API int pdf_surrogate_map(pdf_surrogate *s, unsigned char *states);

/* x f for all flavours, out [n][nflav] FP64: the network on accepted tiles,
 * the FP64 interpolator everywhere else (rejected tiles, outside the grid,
 * invalid points).  *n_fallback (HOST, may be NULL) counts the points that
 * took the interpolator.  Needs an error map; reads the fallback count back,
 * so it synchronises `stream`. */
PDF_API int pdf_surrogate_eval_fallback(pdf_surrogate *s, const pdf_grid *grid, const double *x, const double *q2,
                                        size_t n, double *out, unsigned long long *n_fallback, cudaStream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* PDF_SURROGATE_H */
