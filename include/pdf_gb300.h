/*
 * pdf_gb300.h -- C ABI of the GB300 PDF / alpha_s evaluation library.
 *
 * The library evaluates parton distribution functions x f(x, Q^2) and the
 * strong coupling alpha_s(Q^2) for large batches of query points on one
 * NVIDIA GB300 (sm_103a), following PDFFlow (arXiv:2009.06635):
 *   - Sec. 2.1 / Fig. 1: a PDF object is made once from the tabulated set
 *     (mkPDF) and then queried for one flavour (xfxQ2), all flavours
 *     (xfxQ2_allpid) or alpha_s (alphas_Q2);
 *   - Sec. 2.2: log-bicubic interpolation in (ln x, ln Q^2) of the tabulated
 *     values, Q subgrids split at flavour thresholds interpolated
 *     independently, finite-difference knot tangents that do not reach past
 *     the x edges or a subgrid boundary;
 *   - Fig. 1 (EXTRAPOLATE): continuation outside the grid -- low x and high
 *     Q^2 continue log-linearly from the two outermost knots (linearly when
 *     either value is not positive); low Q^2 continues with the anomalous
 *     dimension gamma = ln(F(1.01 Q2min)/F(Q2min)) / ln 1.01 as
 *     F(Q2min) rho^(gamma rho + 1 - rho), rho = Q^2/Q2min; corners apply the
 *     Q rule at the two lowest x knots, then the low-x rule;
 *   - Sec. 2.3: alpha_s by log-cubic interpolation of (Q^2, alpha_s) nodes,
 *     subgrids split at repeated nodes, constant outside the node range.
 *
 * Conventions for every call:
 *   - Return value: PDF_OK (0) on success, a negative PDF_ERR_* code
 *     otherwise; pdf_last_error() then describes the failure (per thread).
 *     No C++ exception leaves the library: a failed host allocation inside a
 *     call returns PDF_ERR_ALLOC.
 *   - Query and output pointers of the non-"_host" calls are DEVICE memory
 *     owned by the caller; the call enqueues its kernels on `stream`
 *     (0 = the legacy default stream) and returns without waiting.
 *   - "_host" calls take HOST memory (pinned memory gives the overlapped
 *     fast path), copy through device buffers the grid owns, and return only
 *     when the outputs are in host memory.  Such calls on one grid from
 *     several threads are serialised by the grid (as are pdf_mc_integrate
 *     calls, which share the grid's event scratch).
 *   - Arrays are dense and row-major; outputs of the all-flavour calls are
 *     [n][nflav] in the column order the grid was loaded with.
 *   - A query point with x <= 0, x above the last x knot, Q^2 <= 0,
 *     Q^2 = +inf or a NaN coordinate is invalid: its outputs are NaN and the
 *     grid's invalid-point counter is incremented once per point.
 *     No call traps, spins or aborts on any input values.
 *   - n == 0 is valid and launches nothing.
 */
#ifndef PDF_GB300_H
#define PDF_GB300_H

#include <stddef.h>
#include <cuda_runtime_api.h>

#if defined(__GNUC__)
#define PDF_API __attribute__((visibility("default")))
#else
#define PDF_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

enum {
  PDF_OK = 0,
  PDF_ERR_NULL = -1,       /* a required pointer is NULL                      */
  PDF_ERR_GRID = -2,       /* malformed grid descriptor                       */
  PDF_ERR_PID = -3,        /* flavour id not in the grid                      */
  PDF_ERR_CUDA = -4,       /* a CUDA runtime call or kernel launch failed     */
  PDF_ERR_ALLOC = -5,      /* device or host allocation failed                */
  PDF_ERR_ARG = -6,        /* an argument is out of range                     */
  PDF_ERR_NO_ALPHAS = -7   /* the grid was loaded without alpha_s nodes       */
};

/* Size limits of a grid (checked by pdf_load_grid). */
#define PDF_MAX_NX 2048      /* x knots                                        */
#define PDF_MAX_ROWS 1024    /* Q^2 knots over all subgrids (duplicates count) */
#define PDF_MAX_NFLAV 64     /* flavour columns                                */
#define PDF_MAX_NALPHAS 1024 /* alpha_s nodes                                  */

/* Opaque handle: owns device copies of the knots, the values, the staged
 * per-cell tables and the invalid-point counter. */
typedef struct pdf_grid pdf_grid;

/* A PDF set in LHAPDF layout (host memory, read during pdf_load_grid only;
 * the caller keeps ownership).  PDFFlow Sec. 2.1-2.3.
 *   nx, x_knots      strictly increasing, 0 < x <= 1, nx >= 2.
 *   nsub, nq         number of Q subgrids and knots per subgrid (each >= 2).
 *   q2_knots         sum(nq) values, strictly increasing inside a subgrid; the
 *                    first knot of subgrid s+1 equals the last of subgrid s
 *                    (flavour threshold).  Q2max >= 1.01 Q2min is required by
 *                    the low-Q^2 continuation.
 *   nflav, pids      flavour ids of the value columns (PDG; 21 = gluon,
 *                    pid 0 is accepted as an alias of 21 by pdf_xfxq2).
 *   values           [sum(nq)][nx][nflav] tabulated x f(x, Q^2), finite.
 *   na, as_q2, as_vals  alpha_s nodes (na = 0: no alpha_s); as_q2 > 0
 *                    non-decreasing, a repeated value splits subgrids, every
 *                    subgrid has >= 2 nodes. */
typedef struct {
  int nx;
  const double *x_knots;
  int nsub;
  const int *nq;
  const double *q2_knots;
  int nflav;
  const int *pids;
  const double *values;
  int na;
  const double *as_q2;
  const double *as_vals;
} pdf_grid_desc;

/* Validate `desc`, copy it to the device and stage the per-cell tables
 * (logs of the knots, finite-difference tangent weights, bicubic patch
 * coefficients in FP64 and FP32, alpha_s cubic coefficients).  PDFFlow
 * Sec. 2.1 (mkPDF) and 2.2 (data loaded once into device tensors).
 * Synchronous; uses the current CUDA device.  *out receives the handle. */
PDF_API int pdf_load_grid(const pdf_grid_desc *desc, pdf_grid **out);

/* A set of PDF members (replicas of a fit) that share the knots, subgrids
 * and flavours of `desc`: member m's values are member_values[m] laid out as
 * desc->values ([nmem][rows][nx][nflav] host FP64; desc->values is ignored).
 * Every other call evaluates member 0; xfxq2_all_members evaluates all of
 * them.  PDFFlow Sec. 4.3 (multi-member evaluation for fits, Table 2). */
PDF_API int pdf_load_grid_members(const pdf_grid_desc *desc, int nmem, const double *member_values,
                                  pdf_grid **out);
PDF_API int pdf_grid_nmembers(const pdf_grid *grid);

/* LHAPDF6 sets in the "lhagrid1" text format, read directly as PDFFlow
 * Sec. 2.2 does (no conversion step); the alpha_s nodes come from the set's
 * metadata (Sec. 2.3).  A set is a directory NAME/ with NAME.info (YAML:
 * Flavors, AlphaS_Qs, AlphaS_Vals are read; lists may span lines) and
 * NAME_0000.dat, NAME_0001.dat, ... (a YAML header closed by "---", then per
 * Q subgrid: a line of x knots, a line of Q knots in GeV, a line of pids,
 * nx * nq lines of nflav values xf with x the outer loop, and "---").  The
 * subgrids must share the x knots and the flavours.
 *
 * pdf_load_lhapdf: members first_member .. first_member + nmem - 1 of the set
 * in set_dir onto the current device (nmem = 1: pdf_load_grid; nmem > 1:
 * pdf_load_grid_members, every member with the same knots and flavours).
 * Errors: PDF_ERR_NULL, PDF_ERR_ARG (unreadable file, a member range not
 * inside the four-digit file numbers 0..9999), PDF_ERR_GRID (malformed file;
 * the message names the file and the line's subgrid), PDF_ERR_ALLOC (host
 * memory), and those of pdf_load_grid.
 *
 * pdf_lhapdf_read / pdf_lhapdf_desc / pdf_lhapdf_free: the parser alone, on
 * the host (no device work): read one .info + .dat pair into a host object,
 * describe it as a pdf_grid_desc whose arrays point into that object (valid
 * until pdf_lhapdf_free), free it. */
typedef struct pdf_lhapdf_set pdf_lhapdf_set;
PDF_API int pdf_load_lhapdf(const char *set_dir, int first_member, int nmem, pdf_grid **out);
PDF_API int pdf_lhapdf_read(const char *info_path, const char *dat_path, pdf_lhapdf_set **out);
PDF_API int pdf_lhapdf_desc(const pdf_lhapdf_set *set, pdf_grid_desc *desc);
PDF_API int pdf_lhapdf_free(pdf_lhapdf_set *set);

/* Free a handle and all its device memory (NULL is a no-op).  Waits for
 * work the handle's own streams still run. */
PDF_API int pdf_free_grid(pdf_grid *grid);

/* Number of flavour columns and the column index of a pid (-1 if absent). */
PDF_API int pdf_grid_nflav(const pdf_grid *grid);
PDF_API int pdf_grid_pid_column(const pdf_grid *grid, int pid);

/* x f(x, Q^2) of one flavour `pid` at n points: x, q2, out are [n] FP64
 * device arrays.  PDFFlow Sec. 2.1 (xfxQ2), Sec. 2.2. */
PDF_API int xfxq2(const pdf_grid *grid, int pid, const double *x, const double *q2, size_t n,
          double *out, cudaStream_t stream);

/* All flavours at n points: out is [n][nflav] FP64.  PDFFlow (xfxQ2_allpid). */
PDF_API int xfxq2_all_flavours(const pdf_grid *grid, const double *x, const double *q2, size_t n,
                       double *out, cudaStream_t stream);

/* All flavours of all members at n points: out is [nmem][n][nflav] FP64.
 * The cell search, logarithms and weights of a point are computed once and
 * reused for every member.  PDFFlow Sec. 4.3. */
PDF_API int xfxq2_all_members(const pdf_grid *grid, const double *x, const double *q2, size_t n,
                              double *out, cudaStream_t stream);

/* All flavours and alpha_s at the same n points in one pass: out is
 * [n][nflav], alphas_out is [n], FP64 device arrays; ln Q^2 is taken once
 * for both.  Values are those of xfxq2_all_flavours and alphas_q2, bit for
 * bit.  PDFFlow Sec. 2.1 (xfxQ2_allpid), Sec. 2.3 (alphas_Q2).  Errors:
 * PDF_ERR_NULL (alphas_out NULL with n > 0), PDF_ERR_NO_ALPHAS. */
PDF_API int xfxq2_all_flavours_alphas(const pdf_grid *grid, const double *x, const double *q2, size_t n,
                                      double *out, double *alphas_out, cudaStream_t stream);

/* alpha_s(Q^2) at n points, FP64 [n].  PDFFlow Sec. 2.3 (alphas_Q2). */
PDF_API int alphas_q2(const pdf_grid *grid, const double *q2, size_t n, double *out,
              cudaStream_t stream);

/* alpha_s at n scales given as Q in GeV (not Q^2), FP64 [n]: the kernel
 * squares each Q (one rounding) and continues as alphas_q2, so the result
 * equals alphas_q2 at q2 = Q * Q bit for bit.  Q <= 0, NaN, +inf, or a Q
 * whose square overflows, is invalid (NaN out, counter incremented).
 * PDFFlow Sec. 2.1 / Fig. 1 (alphas_Q), Sec. 2.3. */
PDF_API int alphas_q(const pdf_grid *grid, const double *q, size_t n, double *out, cudaStream_t stream);

/* FP32 variants: float inputs and outputs, FP32 arithmetic and accumulation
 * on FP32-rounded patch coefficients; the knot search is exact for the float
 * inputs (the same cell an FP64 search picks) and ln x, ln Q^2 are taken
 * relative to the cell's knot so that no absolute-log rounding enters. */
PDF_API int xfxq2_f32(const pdf_grid *grid, int pid, const float *x, const float *q2, size_t n,
              float *out, cudaStream_t stream);
PDF_API int xfxq2_all_flavours_f32(const pdf_grid *grid, const float *x, const float *q2, size_t n,
                           float *out, cudaStream_t stream);
PDF_API int alphas_q2_f32(const pdf_grid *grid, const float *q2, size_t n, float *out,
                  cudaStream_t stream);
PDF_API int alphas_q_f32(const pdf_grid *grid, const float *q, size_t n, float *out, cudaStream_t stream);
/* FP32 all flavours and alpha_s in one pass (as xfxq2_all_flavours_alphas);
 * bit-identical to xfxq2_all_flavours_f32 and alphas_q2_f32. */
PDF_API int xfxq2_all_flavours_alphas_f32(const pdf_grid *grid, const float *x, const float *q2, size_t n,
                                          float *out, float *alphas_out, cudaStream_t stream);

/* One Monte Carlo event batch in a single launch (PDFFlow Sec. 4.1: the PDF
 * load of a hadronic integrand): for event e, Q^2 = x1[e] x2[e] s, and
 * out[e] = [ xf(x1, Q^2) for all flavours | xf(x2, Q^2) for all flavours |
 * alpha_s(Q^2) ], i.e. out is [n][2 nflav + 1].  The grid needs alpha_s. */
PDF_API int pdf_mc_event(const pdf_grid *grid, const double *x1, const double *x2, double s, size_t n,
                 double *out, cudaStream_t stream);
PDF_API int pdf_mc_event_f32(const pdf_grid *grid, const float *x1, const float *x2, float s, size_t n,
                     float *out, cudaStream_t stream);

/* Monte Carlo integration driven by the PDF load (PDFFlow Sec. 4.1; the
 * VegasFlow use of Sec. 5): events are generated on the device, their
 * flavours and alpha_s evaluated by the fused event kernel, and their weights
 * summed on the device in a fixed order, chunk by chunk.  Events below the
 * s-hat cut (weight zero) are counted but their PDFs are not evaluated.
 *   Event i (global index): u1 = U(z_{2i}), u2 = U(z_{2i+1}), z_k the k-th
 *   output of SplitMix64 seeded with `seed` (Steele, Lea, Flood, OOPSLA 2014:
 *   state seed + (k+1) * 0x9E3779B97F4A7C15 through its 64-bit finaliser),
 *   U(z) = (z >> 11) * 2^-53; ln x_j = ln x_max + u_j (ln x_min - ln x_max),
 *   x_max = the grid's last x knot; s-hat = x1 x2 sqrt_s^2 = Q^2.
 *   Weight (a toy leading-order observable standing in for the paper's
 *   processes, whose matrix elements are not part of this library):
 *     w = L^2 / s-hat * [ sum_{q=1..5} e_q^2 (xf_q(x1) xf_-q(x2) + xf_-q(x1) xf_q(x2))
 *                         + alpha_s(s-hat)^2 xf_g(x1) xf_g(x2) ]   if s-hat >= shat_min,
 *     w = 0 otherwise; L = ln x_max - ln x_min, e_q = -1/3, 2/3, -1/3, 2/3, -1/3
 *     (d, u, s, c, b).  The mean of w estimates the integral over x1, x2 in
 *     [x_min, x_max] of [...] / (x1 x2 s-hat).
 * sums: HOST [3], receives (sum w, sum w^2, sum |w|) over the events
 * [first_event, first_event + n_events).  chunk: events per launch (>= 1).
 * Requires alpha_s and pids 1..5, -1..-5, 21 (PDF_ERR_NO_ALPHAS, PDF_ERR_PID);
 * 0 < x_min < last x knot, sqrt_s > 0, shat_min >= 0 (PDF_ERR_ARG).  The
 * device scratch (chunk x (2 nflav + 2) doubles) belongs to the grid and is
 * reused: calls on one grid must not overlap.  Returns when sums are on the
 * host; the result is bit-reproducible for given (seed, events, chunk). */
typedef struct {
  double sqrt_s;           /* collider energy, GeV */
  double x_min;            /* lower end of the x1, x2 sampling range */
  double shat_min;         /* cut on s-hat, GeV^2 */
  unsigned long long seed; /* SplitMix64 seed */
} pdf_mc_config;
PDF_API int pdf_mc_integrate(const pdf_grid *grid, const pdf_mc_config *cfg, unsigned long long first_event,
                             unsigned long long n_events, size_t chunk, double *sums, cudaStream_t stream);

/* Host-memory variant of xfxq2_all_flavours (end-to-end use: host inputs,
 * host outputs): out is [n][nflav]; if alphas_out is not NULL it receives
 * alpha_s(q2) [n] as well (the grid then needs alpha_s nodes).  Synchronous;
 * see the conventions above. */
PDF_API int xfxq2_all_flavours_host(const pdf_grid *grid, const double *x, const double *q2, size_t n,
                                    double *out, double *alphas_out);

/* No-allocation variant of xfxq2_all_flavours_host (the paper has no
 * counterpart).  For callers that must not have the library allocate device
 * memory: a generator or integrator that calls the PDF inside its own loop,
 * where a cudaMalloc/cudaFree would synchronise the device and stall it; a
 * program whose device memory is wholly managed by another pool or framework;
 * a process that allows no allocation after start-up.  The host variant above
 * allocates its staging buffers on first use; this one stages through a fixed
 * 16 MiB array (2^21 doubles) compiled into the library, which every GPU that
 * loads the library's kernels holds until the process exits.
 *   - n must not exceed 2^21 / (3 + nflav) points (131072 for 13 flavours);
 *     larger batches are rejected with PDF_ERR_ARG (split them).
 *   - x, q2, out (and alphas_out if not NULL) are HOST memory, as for the host
 *     variant; the copies and kernels run on `stream`, and the call returns
 *     when the outputs are in host memory.  It calls no allocator.
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress) and caches it; make that first call on each
 *     device before any stream capture.
 *   - All calls share the one array and it keeps the last call's contents
 *     (each call writes every word it reads, so nothing needs clearing).
 *     Calls whose work overlaps on the GPU -- from several threads or on
 *     several streams of one device -- race on it and must be serialised by
 *     the caller. */
PDF_API int xfxq2_all_flavours_host_noalloc(const pdf_grid *grid, const double *x, const double *q2,
                                            size_t n, double *out, double *alphas_out, cudaStream_t stream);

/* Vector-Jacobian product of xfxq2_all_flavours (growth beyond the paper:
 * gradients for fitting a PDF).  With L = sum_p sum_f cot[p][f] xf_f(x_p, Q2_p):
 *   grad_x[p] = dL/dx_p, grad_q2[p] = dL/dQ2_p        ([n] FP64, either may be NULL);
 *   grad_values[rows][nx][nflav] += dL/d(knot values)  (may be NULL; accumulated
 *                                   with FP64 atomics, so the summation order --
 *                                   and the last bits -- vary between runs).
 * cot is [n][nflav] FP64.  All pointers are device memory; enqueued on
 * `stream`.  Invalid points get NaN gradients and add nothing to
 * grad_values.  A point exactly on the last x (top Q^2) knot gets the
 * one-sided derivative of the last cell.
 * Batches of 2048 points or more (grids with at most 16 flavours and
 * ~65K cells) are sorted by cell on the device first: the call then takes
 * 8 B per point (plus 4 B per cell) of stream-ordered scratch from a memory
 * pool the library keeps per device, and with grad_values up to 16 zeroed
 * copies of grad_values (64 MB at most, fewer where the scratch limit
 * requires) that take the continuation points' knot terms and are added
 * into grad_values at the end; it releases the scratch on `stream`.  If that
 * memory is not available it runs the unsorted kernel instead.  Both
 * paths agree to rounding (the sorted one sums in-grid knot terms per cell
 * in float-float, to ~2^-46 of each knot's own terms). */
PDF_API int xfxq2_all_flavours_vjp(const pdf_grid *grid, const double *x, const double *q2, size_t n,
                                   const double *cot, double *grad_x, double *grad_q2, double *grad_values,
                                   cudaStream_t stream);

/* Replace the grid's knot values with `values` ([rows][nx][nflav] FP64,
 * DEVICE memory) and re-stage the patch coefficients on `stream` (the knots
 * and subgrids stay).  For fitting loops: no host round trip of the values;
 * the call synchronises `stream` once to learn whether the new values keep
 * the float-float contraction of the FP64 path in range.  Work on other
 * streams that reads the grid must be ordered after it by the caller. */
PDF_API int pdf_grid_set_values(pdf_grid *grid, const double *values, cudaStream_t stream);

/* Bound on the device scratch one call may take for a sorted path (the
 * adjoint's, and the FP32 evaluation's for large batches): stream-ordered
 * memory from a pool the library keeps per device.  A call whose scratch
 * would exceed the bound runs its unsorted kernel, which needs none, with the
 * same results to rounding.  Process-wide; default SIZE_MAX (no bound); 0
 * keeps every call off the sorted paths.  Not part of the paper's method. */
PDF_API int pdf_set_scratch_limit(size_t bytes);
PDF_API int pdf_get_scratch_limit(size_t *bytes);

/* Invalid-point counter: read (synchronous) and reset. */
PDF_API int pdf_grid_invalid_count(const pdf_grid *grid, unsigned long long *count);
PDF_API int pdf_grid_reset_invalid_count(pdf_grid *grid);

/* Description of the last error on the calling thread ("" if none). */
PDF_API const char *pdf_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* PDF_GB300_H */
