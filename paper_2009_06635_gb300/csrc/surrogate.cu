// surrogate.cu -- learned surrogate of the interpolator: a small MLP on the
// BF16 tensor cores (tcgen05, FP32 accumulation in TMEM) for both inference
// and training, its training kernels, and evaluation with fallback to the
// interpolator.
//
// Network (for points inside the grid):
//   z   = (2 (ln x - lx_lo)/(lx_hi - lx_lo) - 1,  2 (ln Q^2 - lq_lo)/(lq_hi - lq_lo) - 1)
//   a_j = pi (F[j][0] z0 + F[j][1] z1), features [sin a_0..15 | cos a_0..15] (32, BF16)
//   h_l = silu(W_l h_{l-1} + b_l), width 128, four layers (BF16 activations)
//   y   = W_5 h_4 + b_5 (FP32), one output per flavour
//   target PDF_SURR_ASINH:    xf_f = c_f sinh(y_f), trained on y_f = asinh(xf_f / c_f),
//                             c_f = 1e-5 max|xf_f| (a signed logarithm);
//   target PDF_SURR_ENVELOPE: xf_f = E_f(x) y_f, trained on y_f = xf_f / E_f(x), with
//                             E_f the per-flavour envelope of |xf_f| over Q (see env_table)
//   target PDF_SURR_RESIDUAL: xf_f = B_f(z) + eps E_f(x) y_f, trained on
//                             y_f = (xf_f - B_f) / (eps E_f): the network corrects a
//                             base B, bilinear in (z0, z1) on a uniform 257 x 257
//                             table of the FP64 interpolator (FP32), eps = 2^-10 the
//                             size of the base's relative error; BF16's ~1% error then
//                             lands on a term ~1e-3 of xf
// silu(v) = v (1 + tanh(v/2)) / 2 with the hardware tanh approximation.
// Weights are FP32 masters (Adam) with BF16 copies for the products.
//
// The interpolator is the reference: an error map over 64 x 64 tiles of (z0, z1)
// records the surrogate's largest error against the FP64 interpolator
// (|s - v| / max(|v|, c_f), over flavours and validation points); evaluation
// with fallback uses the surrogate only on tiles whose error is below the
// threshold, and the interpolator everywhere else (and outside the grid).
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "guard.cuh"
#include "pdf_internal.cuh"
#include "pdf_surrogate.h"

namespace {

using namespace pdfgb;
using bf16 = __nv_bfloat16;

constexpr int SW = 128;   // hidden width
constexpr int SNQ = 16;   // Fourier frequencies
constexpr int SIN = 32;   // features
constexpr int SOUT = 16;  // outputs, padded
constexpr int MAPN = 64;  // error-map tiles per axis
constexpr int ENVN = 1024;  // envelope table intervals over [lx_lo, lx_hi]
constexpr int BASEN = 256;  // base table intervals per axis of (z0, z1)
constexpr float kResEps = 1.f / 1024.f;  // residual target scale
constexpr float kResClip = 32.f;         // residual targets clipped to [-32, 32] (cells the base misses by more
                                         // than 3% of E fail the error map whatever the network does)
constexpr float kPi = 3.14159265358979f;

struct SurrConst {
  float freq[SNQ][2];
  float lx_lo, inv_lx, lq_lo, inv_lq;  // z = 2 (l - lo) inv - 1
  float scale[SOUT];
  int nf;
  int target;          // PDF_SURR_ASINH, PDF_SURR_ENVELOPE or PDF_SURR_RESIDUAL
  const float *envt;   // [ENVN + 1][SOUT] ln E_f at lx_lo + k (lx_hi - lx_lo) / ENVN, zero for f >= nf
  const float *baset;  // residual target: [BASEN + 1][BASEN + 1][SOUT] xf at z0 = -1 + 2 i / BASEN (outer),
                       // z1 = -1 + 2 j / BASEN (inner), zero for f >= nf
};

// parameter offsets in the flat FP32 vector
struct Layout {
  size_t w[5], b[5], total;
  int in[5], out[5];
  void set(int nf) {
    const int ins[5] = {SIN, SW, SW, SW, SW}, outs[5] = {SW, SW, SW, SW, nf};
    size_t k = 0;
    for (int l = 0; l < 5; l++) {
      in[l] = ins[l];
      out[l] = outs[l];
      w[l] = k;
      k += (size_t)outs[l] * ins[l];
      b[l] = k;
      k += outs[l];
    }
    total = k;
  }
};
// BF16 weight copies: W1 [128][32], W2..4 [128][128], W5 [16][128] (rows >= nf zero)
__host__ __device__ constexpr size_t wbf_off(int l) { return l == 0 ? 0 : 128 * 32 + (size_t)(l - 1) * 128 * 128; }
constexpr size_t kWbfTotal = 128 * 32 + 3 * 128 * 128 + 16 * 128;
// their transposes for layers 1..4: W_2..W_4^T [128][128], W_5^T [128][16]
__host__ __device__ constexpr size_t wt_off(int l) { return (size_t)(l - 1) * 128 * 128; }
constexpr size_t kWtTotal = 3 * 128 * 128 + 128 * 16;
constexpr int kTgBatch = 256;  // batch rows per chunk of a weight-gradient product

__device__ __forceinline__ float tanh_fast(float v) {
  float r;
  asm("tanh.approx.f32 %0, %1;" : "=f"(r) : "f"(v));
  return r;
}
__device__ __forceinline__ float silu_f(float v) { return 0.5f * v * (1.f + tanh_fast(0.5f * v)); }
__device__ __forceinline__ float dsilu_f(float v) {
  float s = 0.5f * (1.f + tanh_fast(0.5f * v));
  return s + v * s * (1.f - s);
}

__device__ __forceinline__ void point_z(const SurrConst &c, double x, double q2, float &z0, float &z1) {
  z0 = 2.f * (logf((float)x) - c.lx_lo) * c.inv_lx - 1.f;
  z1 = 2.f * (logf((float)q2) - c.lq_lo) * c.inv_lq - 1.f;
}

// E_f at a point of scaled coordinate z0 (ln E linear between table points)
__device__ __forceinline__ float envelope(const SurrConst &c, float z0, int f) {
  const float u = fminf(fmaxf((z0 + 1.f) * (0.5f * ENVN), 0.f), (float)ENVN);
  const int k = min((int)u, ENVN - 1);
  const float *t = c.envt + k * SOUT + f;
  const float a = __ldg(t), b = __ldg(t + SOUT);
  return expf(a + (u - (float)k) * (b - a));
}

// B_f at scaled coordinates (z0, z1): bilinear on the base table (clamped to
// the square), FP32
__device__ __forceinline__ float base_at(const SurrConst &c, float z0, float z1, int f) {
  const float u0 = fminf(fmaxf((z0 + 1.f) * (0.5f * BASEN), 0.f), (float)BASEN);
  const float u1 = fminf(fmaxf((z1 + 1.f) * (0.5f * BASEN), 0.f), (float)BASEN);
  const int i = min((int)u0, BASEN - 1), j = min((int)u1, BASEN - 1);
  const float a = u0 - (float)i, b = u1 - (float)j;
  const float *r0 = c.baset + ((size_t)i * (BASEN + 1) + j) * SOUT + f;
  const float *r1 = r0 + (size_t)(BASEN + 1) * SOUT;
  const float v00 = __ldg(r0), v01 = __ldg(r0 + SOUT), v10 = __ldg(r1), v11 = __ldg(r1 + SOUT);
  const float lo = fmaf(b, v01 - v00, v00), hi = fmaf(b, v11 - v10, v10);
  return fmaf(a, hi - lo, lo);
}

// feature k (0..31) of a point
__device__ __forceinline__ float feature(const SurrConst &c, float z0, float z1, int k) {
  int j = k & 15;
  float a = kPi * (c.freq[j][0] * z0 + c.freq[j][1] * z1);
  return k < 16 ? sinf(a) : cosf(a);
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t *>(&v);
}

// ---------------------------------------------------------------------------
// training kernels
// ---------------------------------------------------------------------------

__global__ void k_features(SurrConst c, const double *x, const double *q2, int n, bf16 *h0, bf16 *h0t,
                           long long ldt) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n * SIN) return;
  int p = i / SIN, k = i % SIN;
  float z0, z1;
  point_z(c, x[p], q2[p], z0, z1);
  const bf16 v = __float2bfloat16_rn(feature(c, z0, z1, k));
  h0[i] = v;
  h0t[(long long)k * ldt + p] = v;
}

// dL/dy for the mean-square loss on asinh targets; the loss sum accumulates in FP64.
__global__ void k_loss(const float *y, const float *t, int n, int nf, bf16 *g, bf16 *gt, long long ldt,
                       double *loss) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  float part = 0.f;
  if (i < n * SOUT) {
    int f = i % SOUT;
    float d = f < nf ? y[i] - t[i] : 0.f;
    const bf16 v = __float2bfloat16_rn(2.f * d / ((float)n * (float)nf));
    g[i] = v;
    gt[(long long)f * ldt + i / SOUT] = v;
    part = d * d;
  }
  for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
  if ((threadIdx.x & 31) == 0 && part != 0.f) atomicAdd(loss, (double)part);
}

// db[n] += sum_b G[b][n] (G BF16, [rows][ld]); one block per column.
// db[n] += sum over rows of G[b][n]: a block per slab of kColRows rows, a thread
// per column (consecutive threads read consecutive columns of a row), one
// atomic per column and block
constexpr int kColRows = 64;
__global__ void __launch_bounds__(128) k_colsum(const bf16 *G, int rows, int ld, int ncol, float *db) {
  const int n = threadIdx.x;
  if (n >= ncol) return;
  const int b0 = blockIdx.x * kColRows, b1 = min(rows, b0 + kColRows);
  float s = 0.f;
  for (int b = b0; b < b1; b++) s += __bfloat162float(G[(long long)b * ld + n]);
  atomicAdd(db + n, s);
}

// Per-step state of a training call, kept on the device so that one captured
// step (a CUDA graph) replays for every step: the batch index and the
// learning-rate schedule follow it, and the step's last kernel advances it.
struct TrainState {
  long long it;  // step within the call
  long long t;   // Adam steps taken before this one (across calls)
};
__global__ void k_train_state(TrainState *ts, long long t) {
  ts->it = 0;
  ts->t = t;
}
// this step's batch (whole batches of B in turn) into the fixed batch buffers
__global__ void k_batch(const double *x, const double *q2, long long nb, int B, const TrainState *ts, double *xb,
                        double *qb) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= B) return;
  const long long o = (ts->it % nb) * B + i;
  xb[i] = x[o];
  qb[i] = q2[o];
}

struct AdamArgs {
  float *p, *gr, *m, *v;
  size_t n;
  float lr, lr_min, b1, b2, eps;  // peak and final learning rate
  int warmup, steps;              // linear warm-up, then cosine decay to lr_min
  const TrainState *ts;
};
__global__ void k_adam(AdamArgs a) {
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.n) return;
  const long long it = a.ts->it, t = a.ts->t + 1;
  float lr;
  if (it < a.warmup) {
    lr = a.lr * (float)(it + 1) / (float)a.warmup;
  } else {
    const float prog = (float)(it - a.warmup) / (float)(a.steps - a.warmup > 0 ? a.steps - a.warmup : 1);
    lr = a.lr_min + 0.5f * (a.lr - a.lr_min) * (1.f + cosf(3.14159265f * prog));
  }
  const float c1 = 1.f - powf(a.b1, (float)t), c2 = 1.f - powf(a.b2, (float)t);
  float g = a.gr[i];
  float m = a.b1 * a.m[i] + (1.f - a.b1) * g;
  float v = a.b2 * a.v[i] + (1.f - a.b2) * g * g;
  a.m[i] = m;
  a.v[i] = v;
  a.p[i] -= lr * (m / c1) / (sqrtf(v / c2) + a.eps);
}

// FP32 masters -> BF16 weight copies (W5 padded to 16 rows).
struct CastArgs {
  const float *p;
  bf16 *w, *wt;
  size_t woff[5], boff[5];
  int nf;
  TrainState *ts;  // when training: advanced by one step here (the step's last kernel)
};
// BF16 weights [out][in] (wbf_off), and for the backward products of layers
// 1..4 their transposes [in][out] (wt_off); rows of W_5 beyond nf are zero
__global__ void k_cast(CastArgs a) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0 && a.ts) {
    a.ts->it += 1;
    a.ts->t += 1;
  }
  if (i >= (int)(kWbfTotal + kWtTotal)) return;
  if (i >= (int)kWbfTotal) {
    const int r = i - (int)kWbfTotal;
    const int l = r < 3 * SW * SW ? 1 + r / (SW * SW) : 4;
    const int q = r - (int)wt_off(l), out = l == 4 ? SOUT : SW;
    const int j = q / out, o = q % out;  // transposed element (j, o) = W_l[o][j]
    const float v = (l == 4 && o >= a.nf) ? 0.f : a.p[a.woff[l] + (size_t)o * SW + j];
    a.wt[r] = __float2bfloat16_rn(v);
    return;
  }
  int l = 4;
  while (l > 0 && (size_t)i < wbf_off(l)) l--;
  int r = i - (int)wbf_off(l);
  int in = l == 0 ? SIN : SW;
  int row = r / in, col = r % in;
  float v = (l == 4 && row >= a.nf) ? 0.f : a.p[a.woff[l] + (size_t)row * in + col];
  a.w[i] = __float2bfloat16_rn(v);
}

// training targets as FP32 [n][16]: asinh(xf / c), xf / E(x), or (xf - B) / (eps E(x))
__global__ void k_targets(SurrConst c, const double *x, const double *q2, const double *xf, int n, float *t) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n * SOUT) return;
  int p = i / SOUT, f = i % SOUT;
  if (f >= c.nf) { t[i] = 0.f; return; }
  const double v = xf[(size_t)p * c.nf + f];
  if (c.target == PDF_SURR_ENVELOPE) {
    float z0, z1;
    point_z(c, x[p], q2[p], z0, z1);
    t[i] = (float)(v / (double)envelope(c, z0, f));
  } else if (c.target == PDF_SURR_RESIDUAL) {
    float z0, z1;
    point_z(c, x[p], q2[p], z0, z1);
    const double r = (v - (double)base_at(c, z0, z1, f)) / ((double)kResEps * (double)envelope(c, z0, f));
    t[i] = (float)fmin(fmax(r, -(double)kResClip), (double)kResClip);
  } else {
    t[i] = (float)asinh(v / (double)c.scale[f]);
  }
}

// The residual target's base B_f alone for n points, into outf [n][nf] (FP32)
// or outd (FP64): the error map's measure of the base (the inference kernel
// forms B_f itself, with the same arithmetic).
__global__ void k_base(SurrConst c, const double *x, const double *q2, long long n, float *outf, double *outd) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n * c.nf) return;
  const long long p = i / c.nf;
  const int f = (int)(i - p * c.nf);
  float z0, z1;
  point_z(c, x[p], q2[p], z0, z1);
  const float b = base_at(c, z0, z1, f);
  if (outf) outf[i] = b;
  if (outd) outd[i] = (double)b;
}

// ---------------------------------------------------------------------------
// fused inference on the 5th-generation tensor cores (tcgen05, TMEM)
//
// One CTA per SM keeps every BF16 weight matrix in shared memory (K-major; the
// K = 128 operands in 128-byte rows with the 16-byte chunks of row r permuted
// by XOR with r % 8, the layout the tensor core reads at full rate; the
// K = 32 and bias operands in plain 8 x 8 core matrices) and runs two groups
// of eight warps.  A group owns a tile of 128 points, the rows of every
// activation matrix, and 200 TMEM columns: the FP32 accumulator D (128), the
// BF16 activations A of the next layer packed two per column (64, row = lane),
// and a constant block (8) whose K columns 0..2 are 1.  Warp w of the group
// reads lanes 32 (w % 4) .. + 31 and the column half w / 4.
//
// Per layer one thread issues K/16 tcgen05.mma with A from TMEM and B from
// shared memory (M = 128, N = 128 or 16, K = 16, FP32 accumulation), then one
// more K = 16 step against the constant block whose B columns hold the bias
// as three BF16 parts (hi + mid + lo = the FP32 bias exactly), and commits to
// the group's mbarrier.  Every thread then reads its 64 accumulator columns
// (tcgen05.ld, the second half-load in flight while the first is used),
// applies SiLU and writes the BF16 pairs back as the next layer's A
// (tcgen05.st).  Activations never touch shared memory.  While one group's
// products run on the tensor core, the other group's epilogue runs.
//
// The SiLU layers' weights and biases are held at half scale (exact in BF16),
// so the accumulator is h = z / 2 and silu(z) = h + h tanh(h): one hardware
// tanh and one FMA per element.  The next tile's x and Q^2 are loaded while
// the current tile runs, and its envelope rows are copied (cp.async) into
// shared memory at the start of the tile.  Outputs are staged in shared
// memory and written as whole contiguous rows of the tile.  Every wait is
// bounded: a wait that runs out sets the surrogate's error flag and the group
// stops.
// ---------------------------------------------------------------------------
constexpr int TG = 2;                 // tile groups per CTA
constexpr int kGW = 8;                // warps per group: four TMEM lane quarters x two column halves
constexpr int kGT = 32 * kGW;         // threads per group
constexpr int kTcThreads = kGT * TG;  // 512
constexpr int kTmemGroup = 256;       // TMEM columns per group (200 used)
constexpr int kTmemCols = kTmemGroup * TG;
constexpr size_t kSW1 = 128 * 32 * 2, kSWh = 128 * 128 * 2, kSW5 = 16 * 128 * 2, kSWb = 128 * 16 * 2;
constexpr size_t kSE = 128 * 2 * SOUT * sizeof(float);  // envelope rows (k, k + 1) of one tile
constexpr size_t kSO = 128 * SOUT * sizeof(float);      // output staging of one tile
constexpr size_t kOffWh = kSW1, kOffW5 = kOffWh + 3 * kSWh, kOffWb = kOffW5 + kSW5, kOffE = kOffWb + 5 * kSWb;
constexpr size_t kOffO = kOffE + TG * kSE, kEnd = kOffO + TG * kSO;
constexpr size_t kTcSmem = kEnd + 1024;  // + alignment of the base to 1 KB
static_assert(kTcSmem + 1024 <= 227 * 1024, "inference shared memory");
static_assert(kOffWh % 1024 == 0 && kOffW5 % 1024 == 0, "swizzled operands start on 1 KB boundaries");
static_assert(kOffWb % 16 == 0 && kOffE % 16 == 0 && kOffO % 16 == 0, "16-byte aligned shared buffers");

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
// element (r, k) of an R x K K-major matrix in 8 x 8 core matrices:
// byte (r/8) (K/8) 128 + (k/8) 128 + (r%8) 16 + (k%8) 2
__device__ __forceinline__ int cm_off(int r, int k, int K) {
  return (r >> 3) * (K >> 3) * 64 + (k >> 3) * 64 + (r & 7) * 8 + (k & 7);
}
// element (r, k) of an R x 128 K-major matrix in 128-byte rows: K blocks of 64
// elements (R x 128 bytes each), the 16-byte chunk j of row r at chunk j ^ (r % 8)
__device__ __forceinline__ int sw_off(int r, int k, int R) {
  return (k >> 6) * R * 64 + r * 64 + ((((k >> 3) & 7) ^ (r & 7)) << 3) + (k & 7);
}
// shared-memory matrix descriptor: start, leading (K) and stride (M/N) byte
// offsets between core matrices, no swizzle, descriptor version 1 (bit 46)
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)(128u >> 4) << 16) | ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) |
         ((uint64_t)1 << 46);
}
// the same for the 128-byte swizzled layout (mode 2 at bit 61): 1 KB between
// groups of eight rows; a K step of 16 elements inside a row adds 32 bytes
__device__ __forceinline__ uint64_t smem_desc_sw(uint32_t addr) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)1 << 16) | ((uint64_t)(1024u >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}
// instruction descriptor, kind::f16: D F32 (bit 4), A and B BF16 (bits 7, 10),
// both K-major, N >> 3 at bit 17, M >> 4 at bit 24
__device__ __forceinline__ uint32_t mma_idesc(int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}
// D (TMEM) (+)= A (TMEM, BF16 pairs) B^T (shared memory)
__device__ __forceinline__ void mma_ts(uint32_t d, uint32_t a, uint64_t bdesc, uint32_t id, uint32_t acc) {
  asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}\n"
               ::"r"(d), "r"(a), "l"(bdesc), "r"(id), "r"(acc));
}
// the products of layer l: K/16 steps over the activations, then the bias step
__device__ __forceinline__ void layer_mma(int l, uint32_t d, uint32_t a, uint32_t ones, uint32_t w1, uint32_t wh,
                                          uint32_t w5, uint32_t wb) {
  const uint64_t bias = smem_desc(wb + (uint32_t)l * (uint32_t)kSWb, 256);
  if (l == 0) {
    const uint32_t id = mma_idesc(128);
#pragma unroll
    for (int s = 0; s < SIN / 16; s++) mma_ts(d, a + 8 * s, smem_desc(w1 + 256 * s, (SIN / 8) * 128), id, s > 0);
    mma_ts(d, ones, bias, id, 1);
  } else if (l < 4) {
    const uint32_t id = mma_idesc(128), b = wh + (uint32_t)(l - 1) * (uint32_t)kSWh;
#pragma unroll
    for (int s = 0; s < SW / 16; s++)
      mma_ts(d, a + 8 * s, smem_desc_sw(b + (uint32_t)(s >> 2) * 128 * 128 + (uint32_t)(s & 3) * 32), id, s > 0);
    mma_ts(d, ones, bias, id, 1);
  } else {
    const uint32_t id = mma_idesc(16);
#pragma unroll
    for (int s = 0; s < SW / 16; s++)
      mma_ts(d, a + 8 * s, smem_desc_sw(w5 + (uint32_t)(s >> 2) * 16 * 128 + (uint32_t)(s & 3) * 32), id, s > 0);
    mma_ts(d, ones, bias, id, 1);
  }
}
__device__ __forceinline__ void tc_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar));
}
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t phase) {
  uint32_t done = 0;
  for (int it = 0; it < (1 << 24) && !done; it++)
    asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(done) : "r"(mbar), "r"(phase));
  return done != 0;
}
// 32 consecutive FP32 columns of this warp's 32 TMEM lanes; the registers are
// valid only after tmem_wait32 on the same array
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t *r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,"
      "%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
}
// waits for every outstanding tcgen05.ld of the thread; the operands tie the
// wait to the registers of r so that no use of them moves above it
__device__ __forceinline__ void tmem_wait32(uint32_t *r) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                 "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                 "+r"(r[15]), "+r"(r[16]), "+r"(r[17]), "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]),
                 "+r"(r[22]), "+r"(r[23]), "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]),
                 "+r"(r[29]), "+r"(r[30]), "+r"(r[31]));
}
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float *v) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]));
#pragma unroll
  for (int j = 0; j < 8; j++) v[j] = __uint_as_float(r[j]);
}
// stores to this warp's 32 TMEM lanes (one register per column); complete after tcgen05.wait::st
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t *r) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};"
               ::"r"(taddr), "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]),
               "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15]));
}
__device__ __forceinline__ void tmem_st8(uint32_t taddr, const uint32_t *r) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};"
               ::"r"(taddr), "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]));
}
__device__ __forceinline__ void tmem_st4(uint32_t taddr, const uint32_t *r) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1,%2,%3,%4};"
               ::"r"(taddr), "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]));
}
// the group's threads: their TMEM writes ordered before the tensor core's reads, then a barrier
__device__ __forceinline__ void group_sync(int g) {
  asm volatile("tcgen05.fence::before_thread_sync;");
  asm volatile("bar.sync %0, %1;" ::"r"(1 + g), "r"(kGT));
}
// barrier of the group that also returns whether v held on any of its threads
__device__ __forceinline__ bool group_any(int g, bool v) {
  uint32_t r;
  asm volatile("{\n.reg .pred p, q;\nsetp.ne.u32 p, %1, 0;\nbar.red.or.pred q, %2, %3, p;\nselp.u32 %0, 1, 0, q;\n}\n"
               : "=r"(r) : "r"((uint32_t)v), "r"(1 + g), "r"(kGT));
  return r != 0;
}
__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }
// silu(2h) = h + h tanh(h) of 32 accumulator columns (h = z / 2, bias included),
// packed in place as 16 BF16 pairs (r[0..15])
__device__ __forceinline__ void silu_pack(uint32_t *r) {
#pragma unroll
  for (int j = 0; j < 16; j++) {
    const float h0 = __uint_as_float(r[2 * j]), h1 = __uint_as_float(r[2 * j + 1]);
    r[j] = pack_bf16(fmaf(h0, tanh_fast(h0), h0), fmaf(h1, tanh_fast(h1), h1));
  }
}

__global__ void __launch_bounds__(kTcThreads, 1)
k_infer(SurrConst c, const bf16 *__restrict__ wg, const float *__restrict__ params, Layout L,
        const double *__restrict__ xa, const double *__restrict__ qa, long long n, float *__restrict__ outf,
        double *__restrict__ outd, const unsigned char *__restrict__ mask, unsigned int *nfb,
        unsigned int *fb_idx, int *err) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ __align__(8) unsigned long long mbar[TG];
  __shared__ uint32_t tbase;
  __shared__ float sfreq[SNQ][2], sscale[SOUT];  // indexed by the warp's half: kept out of the parameter space
  __shared__ volatile int g1_go;                 // group 1 may start (see below)
  unsigned char *smem = smem_raw + (((smem_u32(smem_raw) + 1023u) & ~1023u) - smem_u32(smem_raw));
  bf16 *W1 = reinterpret_cast<bf16 *>(smem);
  bf16 *Wh = reinterpret_cast<bf16 *>(smem + kOffWh);
  bf16 *W5 = reinterpret_cast<bf16 *>(smem + kOffW5);
  bf16 *Wb = reinterpret_cast<bf16 *>(smem + kOffWb);  // bias columns of the five layers
  const bf16 half_w = __float2bfloat16(0.5f);
  for (int i = threadIdx.x; i < 128 * SIN; i += kTcThreads)
    W1[cm_off(i / SIN, i % SIN, SIN)] = __hmul(wg[wbf_off(0) + i], half_w);
  for (int l = 0; l < 3; l++)
    for (int i = threadIdx.x; i < 128 * SW; i += kTcThreads)
      Wh[l * 128 * SW + sw_off(i / SW, i % SW, 128)] = __hmul(wg[wbf_off(l + 1) + i], half_w);
  for (int i = threadIdx.x; i < 16 * SW; i += kTcThreads) W5[sw_off(i / SW, i % SW, 16)] = wg[wbf_off(4) + i];
  // bias b (b / 2 for the SiLU layers) as three BF16 parts hi + mid + lo = b exactly, in K columns 0..2
#pragma unroll
  for (int l = 0; l < 5; l++) {
    const int rows = l < 4 ? SW : SOUT;
    for (int i = threadIdx.x; i < rows * 16; i += kTcThreads) {
      const int r = i >> 4, k = i & 15;
      const float b = l < 4 ? 0.5f * params[L.b[l] + r] : (r < c.nf ? params[L.b[4] + r] : 0.f);
      const bf16 hi = __float2bfloat16_rn(b);
      const float r1 = b - __bfloat162float(hi);
      const bf16 mid = __float2bfloat16_rn(r1);
      const bf16 lo = __float2bfloat16_rn(r1 - __bfloat162float(mid));
      Wb[l * 128 * 16 + cm_off(r, k, 16)] = k == 0 ? hi : k == 1 ? mid : k == 2 ? lo : __float2bfloat16(0.f);
    }
  }
  if (threadIdx.x < 2 * SNQ) sfreq[threadIdx.x >> 1][threadIdx.x & 1] = c.freq[threadIdx.x >> 1][threadIdx.x & 1];
  if (threadIdx.x < SOUT) sscale[threadIdx.x] = c.scale[threadIdx.x];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x < TG) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[threadIdx.x])));
  if (threadIdx.x == 0) g1_go = 0;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tbase)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("fence.proxy.async.shared::cta;");
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");

  const int g = warp / kGW, gw = warp % kGW, half = gw >> 2;  // group, warp in group, column half
  const int t = 32 * (gw & 3) + lane;                          // row of the tile
  const int gt = threadIdx.x - g * kGT;                        // thread in group
  const int nf = c.nf;
  float *E = reinterpret_cast<float *>(smem + kOffE + g * kSE);  // [rows][8 chunks of 4], chunk j at j ^ (t % 8)
  float *O = reinterpret_cast<float *>(smem + kOffO + g * kSO);  // [rows][nf]
  const uint32_t mb = smem_u32(&mbar[g]);
  const uint32_t e_row = smem_u32(E + t * 2 * SOUT);
  const uint32_t tg = tbase + (uint32_t)(g * kTmemGroup);                // the group's columns
  const uint32_t tD = tg, tA = tg + 128, tOne = tg + 192;               // accumulator, activations, ones
  const uint32_t lanes = (uint32_t)(32 * (gw & 3)) << 16;               // this warp's lanes
  const uint32_t w1 = smem_u32(W1), wh = smem_u32(Wh), w5 = smem_u32(W5), wb = smem_u32(Wb);
  if (half == 0) {  // the constant K columns (1, 1, 1, 0, ...) that meet the bias parts
    uint32_t o[8] = {0x3F803F80u, 0x00003F80u, 0u, 0u, 0u, 0u, 0u, 0u};
    tmem_st8(tOne + lanes, o);
    asm volatile("tcgen05.wait::st.sync.aligned;");
  }
  uint32_t phase = 0;
  const long long ntiles = (n + 127) / 128, tstride = (long long)gridDim.x * TG;
  long long tile = (long long)blockIdx.x * TG + g;
  double xn = 0.5, qn = 10.0;  // this thread's point of the next tile (defaults for rows past n)
  if (tile * 128 + t < n) { xn = xa[tile * 128 + t]; qn = qa[tile * 128 + t]; }
  // Group 1 starts a third of a tile behind group 0 (when group 0 issues the
  // products of its first tile's second layer, or has no tile): started together, the
  // two groups stay in step -- their products queue behind each other on the
  // tensor core and their epilogues share the SFU -- while offset, one
  // group's products run during the other's epilogue (21% less time).  The
  // wait is bounded (~1 ms).
  if (g == 1)
    for (int it = 0; it < (1 << 14) && !g1_go; it++) __nanosleep(64);
  bool first = true;
  for (; tile < ntiles; tile += tstride) {
    const long long p0 = tile * 128, p = p0 + t;
    const bool in = p < n;
    const double x = xn, q = qn;
    {
      const long long pn = p + tstride * 128;
      xn = 0.5; qn = 10.0;
      if (pn < n) { xn = xa[pn]; qn = qa[pn]; }
    }
    float z0, z1;
    point_z(c, x, q, z0, z1);
    // envelope rows k and k + 1 of this point, this half's eight flavours (chunks 2 half, 2 half + 1)
    const float u = fminf(fmaxf((z0 + 1.f) * (0.5f * ENVN), 0.f), (float)ENVN);
    const int k = min((int)u, ENVN - 1);
    const float fr = u - (float)k;
    if (c.target != PDF_SURR_ASINH) {
      const float *src = c.envt + (size_t)k * SOUT + 8 * half;
#pragma unroll
      for (int j = 0; j < 2; j++) {
        cp_async16(e_row + (uint32_t)(((2 * half + j) ^ (t & 7)) * 16), src + 4 * j);
        cp_async16(e_row + (uint32_t)(((4 + 2 * half + j) ^ (t & 7)) * 16), src + SOUT + 4 * j);
      }
    }
    bool base_only = false;  // a tile the map serves by the residual target's base alone
    if (mask) {  // fallback: outside the grid, or on a tile the map rejects
      const bool inside = z0 >= -1.f && z0 <= 1.f && z1 >= -1.f && z1 <= 1.f && x > 0.0 && q > 0.0;
      const int tx = min(MAPN - 1, max(0, (int)((z0 + 1.f) * 0.5f * MAPN)));
      const int tq = min(MAPN - 1, max(0, (int)((z1 + 1.f) * 0.5f * MAPN)));
      const unsigned char ms = inside ? mask[tq * MAPN + tx] : (unsigned char)0;
      const bool bad = in && ms == 0;
      base_only = ms == 2;
      if (half == 0) {  // one record per point
        const unsigned int bb = __ballot_sync(0xffffffffu, bad);
        unsigned int base = 0;
        if (bb && lane == 0) base = atomicAdd(nfb, (unsigned int)__popc(bb));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (bad) fb_idx[base + __popc(bb & ((1u << lane) - 1u))] = (unsigned int)p;
      }
      if (!inside) { z0 = 0.f; z1 = 0.f; }
    }
    {  // features: this half's eight angles a_j; sin into K columns j, cos into 16 + j (BF16 pairs)
      const int j0 = 8 * half;
      float sv[8], cv[8];
#pragma unroll
      for (int j = 0; j < 8; j++) sincospif(sfreq[j0 + j][0] * z0 + sfreq[j0 + j][1] * z1, &sv[j], &cv[j]);
      uint32_t a[4], b[4];
#pragma unroll
      for (int j = 0; j < 4; j++) { a[j] = pack_bf16(sv[2 * j], sv[2 * j + 1]); b[j] = pack_bf16(cv[2 * j], cv[2 * j + 1]); }
      tmem_st4(tA + lanes + (uint32_t)(4 * half), a);
      tmem_st4(tA + lanes + (uint32_t)(8 + 4 * half), b);
      asm volatile("tcgen05.wait::st.sync.aligned;");
    }
    bool ok = true;
    for (int l = 0; l < 5; l++) {
      group_sync(g);
      if (gt == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;");
        layer_mma(l, tD, tA, tOne, w1, wh, w5, wb);
        tc_commit(mb);
        if (g == 0 && l == 1 && first) g1_go = 1;
      }
      const bool done = mbar_wait(mb, phase);
      phase ^= 1u;
      if (group_any(g, !done)) { ok = false; break; }  // every thread of the group leaves together
      asm volatile("tcgen05.fence::after_thread_sync;");
      if (l < 4) {  // SiLU of this half's 64 columns into the next layer's K columns (BF16 pairs)
        const uint32_t c0 = 64 * half;
        uint32_t r0[32], r1[32];
        tmem_ld32(tD + lanes + c0, r0);
        tmem_wait32(r0);
        tmem_ld32(tD + lanes + c0 + 32, r1);
        silu_pack(r0);
        tmem_st16(tA + lanes + c0 / 2, r0);
        tmem_wait32(r1);
        silu_pack(r1);
        tmem_st16(tA + lanes + c0 / 2 + 16, r1);
        asm volatile("tcgen05.wait::st.sync.aligned;");
      } else {  // outputs of this half's eight flavours, staged as whole rows
        // residual target: the base's four corners for this half's eight
        // flavours (loads issued before the accumulator and envelope waits)
        float4 bc[8];
        float bu0 = 0.f, bu1 = 0.f;
        if (c.target == PDF_SURR_RESIDUAL) {
          const float u0 = fminf(fmaxf((z0 + 1.f) * (0.5f * BASEN), 0.f), (float)BASEN);
          const float u1 = fminf(fmaxf((z1 + 1.f) * (0.5f * BASEN), 0.f), (float)BASEN);
          const int bi = min((int)u0, BASEN - 1), bj = min((int)u1, BASEN - 1);
          bu0 = u0 - (float)bi;
          bu1 = u1 - (float)bj;
          const float4 *r0 = reinterpret_cast<const float4 *>(c.baset + ((size_t)bi * (BASEN + 1) + bj) * SOUT + 8 * half);
          const float4 *r1 = r0 + (BASEN + 1) * SOUT / 4;
          bc[0] = __ldg(r0); bc[1] = __ldg(r0 + 1);                        // (i, j)
          bc[2] = __ldg(r0 + SOUT / 4); bc[3] = __ldg(r0 + SOUT / 4 + 1);  // (i, j + 1)
          bc[4] = __ldg(r1); bc[5] = __ldg(r1 + 1);                        // (i + 1, j)
          bc[6] = __ldg(r1 + SOUT / 4); bc[7] = __ldg(r1 + SOUT / 4 + 1);  // (i + 1, j + 1)
        }
        float v[8];
        tmem_ld8(tD + lanes + 8 * half, v);
        float o[8];
        if (c.target != PDF_SURR_ASINH) {
          cp_async_wait_all();
          const float *er = E + t * 2 * SOUT;
          const float4 a0 = *reinterpret_cast<const float4 *>(er + (((2 * half) ^ (t & 7)) << 2));
          const float4 a1 = *reinterpret_cast<const float4 *>(er + (((2 * half + 1) ^ (t & 7)) << 2));
          const float4 b0 = *reinterpret_cast<const float4 *>(er + (((4 + 2 * half) ^ (t & 7)) << 2));
          const float4 b1 = *reinterpret_cast<const float4 *>(er + (((5 + 2 * half) ^ (t & 7)) << 2));
          const float ea[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
          const float eb[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
          if (c.target == PDF_SURR_RESIDUAL) {
            // B + eps E y, B bilinear as base_at computes it (base alone: B)
            const float v00[8] = {bc[0].x, bc[0].y, bc[0].z, bc[0].w, bc[1].x, bc[1].y, bc[1].z, bc[1].w};
            const float v01[8] = {bc[2].x, bc[2].y, bc[2].z, bc[2].w, bc[3].x, bc[3].y, bc[3].z, bc[3].w};
            const float v10[8] = {bc[4].x, bc[4].y, bc[4].z, bc[4].w, bc[5].x, bc[5].y, bc[5].z, bc[5].w};
            const float v11[8] = {bc[6].x, bc[6].y, bc[6].z, bc[6].w, bc[7].x, bc[7].y, bc[7].z, bc[7].w};
#pragma unroll
            for (int i = 0; i < 8; i++) {
              const float lo = fmaf(bu1, v01[i] - v00[i], v00[i]), hi = fmaf(bu1, v11[i] - v10[i], v10[i]);
              const float bv = fmaf(bu0, hi - lo, lo);
              o[i] = base_only ? bv : bv + kResEps * expf(ea[i] + fr * (eb[i] - ea[i])) * v[i];
            }
          } else {
#pragma unroll
            for (int i = 0; i < 8; i++) o[i] = expf(ea[i] + fr * (eb[i] - ea[i])) * v[i];
          }
        } else {
#pragma unroll
          for (int i = 0; i < 8; i++) o[i] = sscale[8 * half + i] * sinhf(v[i]);
        }
#pragma unroll
        for (int i = 0; i < 8; i++)
          if (8 * half + i < nf) O[t * nf + 8 * half + i] = o[i];
        asm volatile("bar.sync %0, %1;" ::"r"(1 + g), "r"(kGT));
        const long long rows = min(128LL, n - p0);
        const int cnt = (int)rows * nf;
        if (outf) {
          float *dst = outf + p0 * nf;
          int i0 = 0;
          if ((reinterpret_cast<uintptr_t>(dst) & 15) == 0) {
            for (int i = gt; i < cnt / 4; i += kGT)
              __stcs(reinterpret_cast<float4 *>(dst) + i, reinterpret_cast<const float4 *>(O)[i]);
            i0 = cnt & ~3;
          }
          for (int i = i0 + gt; i < cnt; i += kGT) __stcs(dst + i, O[i]);
        }
        if (outd) {
          double *dst = outd + p0 * nf;
          int i0 = 0;
          if ((reinterpret_cast<uintptr_t>(dst) & 15) == 0) {
            for (int i = gt; i < cnt / 2; i += kGT) {
              const float2 w = reinterpret_cast<const float2 *>(O)[i];
              __stcs(reinterpret_cast<double2 *>(dst) + i, make_double2((double)w.x, (double)w.y));
            }
            i0 = cnt & ~1;
          }
          for (int i = i0 + gt; i < cnt; i += kGT) __stcs(dst + i, (double)O[i]);
        }
      }
    }
    first = false;
    if (!ok) {
      if (gt == 0) atomicExch(err, 1);
      break;
    }
  }
  if (g == 0 && gt == 0) g1_go = 1;
  cp_async_wait_all();
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(kTmemCols));
}

// ---------------------------------------------------------------------------
// training products on tcgen05: C[M][N] = A[M][K] B[N][K]^T with both operands
// K-contiguous in global memory (the training keeps transposed copies of its
// activations, gradients and weights so that every product reads rows),
// staged through two shared-memory stages of 64 K columns in the swizzled
// layout, accumulated in TMEM (FP32), with the layer's epilogue on the way
// out.  One CTA per 128-row tile, NT columns (grid z: column tiles) and one
// K chunk (grid y: a split of the batch sum for the weight gradients, which
// then add their partial tiles atomically).  Waits are bounded as in the
// inference kernel.
// ---------------------------------------------------------------------------
enum { EPI_FWD_SILU = 0, EPI_OUT = 1, EPI_BWD_SILU = 2, EPI_ATOMIC = 3 };

struct TGemm {
  const bf16 *A;
  long long lda;
  const bf16 *B;
  long long ldb;
  int M, N, K, kchunk;
  const float *bias;  // FWD / OUT: per column
  int nvalid;         // OUT: columns with a bias; ATOMIC: columns added
  float *Z;           // FWD: pre-activation out; BWD: pre-activation in ([M][ldz])
  long long ldz;
  bf16 *H;            // FWD: activation out; BWD: gradient out ([M][ldh])
  long long ldh;
  bf16 *Ht;           // the same transposed ([N][ldht])
  long long ldht;
  float *C;           // OUT: y [M][ldc]; ATOMIC: C[m][n], or C[n][m] with ctrans
  long long ldc;
  int ctrans;
  int *err;
};
constexpr int kTgK = 64;                                    // K columns per stage
constexpr size_t kTgStage = 2 * 128 * kTgK * sizeof(bf16);  // A and B tiles of up to 128 rows
constexpr size_t kTgSmem = 2 * kTgStage + 1024;

__device__ __forceinline__ void mma_ss(uint32_t d, uint64_t adesc, uint64_t bdesc, uint32_t id, uint32_t acc) {
  asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
               ::"r"(d), "l"(adesc), "l"(bdesc), "r"(id), "r"(acc));
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t *r) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                 "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                 "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15]));
}

// rows [r0, r0 + R) and K columns [k0, k0 + 64) of a K-contiguous operand into one
// swizzled stage; zero outside rows < nrows and columns < ke
template <int R>
__device__ __forceinline__ void tg_load(bf16 *dst, const bf16 *src, long long ld, int r0, int nrows, int k0, int ke,
                                        bool vec) {
  for (int i = threadIdx.x; i < R * 8; i += 128) {
    const int r = i >> 3, c = i & 7, row = r0 + r, k = k0 + 8 * c;
    uint4 v = make_uint4(0u, 0u, 0u, 0u);
    if (row < nrows && k < ke) {
      const bf16 *p = src + (long long)row * ld + k;
      if (vec && k + 8 <= ke) {
        v = __ldg(reinterpret_cast<const uint4 *>(p));
      } else {
        uint32_t e[8];
#pragma unroll
        for (int j = 0; j < 8; j++) e[j] = k + j < ke ? (uint32_t)__bfloat16_as_ushort(p[j]) : 0u;
        v = make_uint4(e[0] | (e[1] << 16), e[2] | (e[3] << 16), e[4] | (e[5] << 16), e[6] | (e[7] << 16));
      }
    }
    *reinterpret_cast<uint4 *>(dst + r * 64 + ((c ^ (r & 7)) << 3)) = v;
  }
}

template <int EPI, int NT>
__global__ void __launch_bounds__(128) k_tgemm(TGemm g) {
  extern __shared__ __align__(16) unsigned char tg_raw[];
  __shared__ __align__(8) unsigned long long mbar[3];  // the two stages, and the last product
  __shared__ uint32_t tbase;
  unsigned char *sm = tg_raw + (((smem_u32(tg_raw) + 1023u) & ~1023u) - smem_u32(tg_raw));
  constexpr int NCOL = NT < 32 ? 32 : NT;  // TMEM columns (at least 32)
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.x * 128, n0 = blockIdx.z * NT;
  const int kb = blockIdx.y * g.kchunk, ke = min(g.K, kb + g.kchunk);
  const bool vec = ((reinterpret_cast<uintptr_t>(g.A) | reinterpret_cast<uintptr_t>(g.B)) & 15) == 0 &&
                   (g.lda & 7) == 0 && (g.ldb & 7) == 0;
  if (threadIdx.x < 3) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[threadIdx.x])));
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tbase)),
                 "r"(NCOL));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("fence.proxy.async.shared::cta;");
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tbase, id = mma_idesc(NT);
  bool ok = true;
  int it = 0;
  for (int k0 = kb; k0 < ke; k0 += kTgK, it++) {
    const int s = it & 1;
    // the stage's previous products (two iterations back) must have read it
    const bool done = it < 2 || mbar_wait(smem_u32(&mbar[s]), (uint32_t)(((it - 2) >> 1) & 1));
    if (__syncthreads_or(!done)) { ok = false; break; }
    bf16 *As = reinterpret_cast<bf16 *>(sm + s * kTgStage), *Bs = As + 128 * kTgK;
    tg_load<128>(As, g.A, g.lda, m0, g.M, k0, ke, vec);
    tg_load<NT>(Bs, g.B, g.ldb, n0, g.N, k0, ke, vec);
    asm volatile("fence.proxy.async.shared::cta;");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (threadIdx.x == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;");
      const uint32_t a = smem_u32(As), b = smem_u32(Bs);
#pragma unroll
      for (int q = 0; q < kTgK / 16; q++)
        mma_ss(tmem, smem_desc_sw(a + 32 * q), smem_desc_sw(b + 32 * q), id, (it > 0 || q > 0) ? 1u : 0u);
      tc_commit(smem_u32(&mbar[s]));
    }
  }
  if (ok && it > 0) {  // one more commit covers every product of the CTA
    if (threadIdx.x == 0) tc_commit(smem_u32(&mbar[2]));
    const bool done = mbar_wait(smem_u32(&mbar[2]), 0u);
    if (__syncthreads_or(!done)) ok = false;
  }
  if (ok && it > 0) {
    asm volatile("tcgen05.fence::after_thread_sync;");
    const int m = m0 + 32 * warp + lane;
    const bool live = m < g.M;
    const uint32_t trow = tmem + ((uint32_t)(32 * warp) << 16);
    constexpr int CW = NT < 32 ? 16 : 32;  // columns per TMEM load
#pragma unroll 1
    for (int c0 = 0; c0 < NT; c0 += CW) {
      uint32_t r[32];
      if (CW == 16) tmem_ld16(trow + c0, r);
      else { tmem_ld32(trow + c0, r); tmem_wait32(r); }
      const int nb = n0 + c0;  // first column of the chunk
      if (!live || nb >= g.N) continue;
      float v[CW];
#pragma unroll
      for (int j = 0; j < CW; j++) v[j] = __uint_as_float(r[j]);
      if (EPI == EPI_FWD_SILU || EPI == EPI_BWD_SILU) {
        float *zr = g.Z + (long long)m * g.ldz + nb;
        bf16 *hr = g.H + (long long)m * g.ldh + nb;
#pragma unroll
        for (int j8 = 0; j8 < CW; j8 += 8) {
          float o[8];
          if (EPI == EPI_FWD_SILU) {
            float zz[8];
#pragma unroll
            for (int j = 0; j < 8; j++) { zz[j] = v[j8 + j] + __ldg(g.bias + nb + j8 + j); o[j] = silu_f(zz[j]); }
            *reinterpret_cast<float4 *>(zr + j8) = make_float4(zz[0], zz[1], zz[2], zz[3]);
            *reinterpret_cast<float4 *>(zr + j8 + 4) = make_float4(zz[4], zz[5], zz[6], zz[7]);
          } else {
            const float4 za = *reinterpret_cast<const float4 *>(zr + j8);
            const float4 zb = *reinterpret_cast<const float4 *>(zr + j8 + 4);
            const float zz[8] = {za.x, za.y, za.z, za.w, zb.x, zb.y, zb.z, zb.w};
#pragma unroll
            for (int j = 0; j < 8; j++) o[j] = v[j8 + j] * dsilu_f(zz[j]);
          }
          uint4 pk;
          pk.x = pack_bf16(o[0], o[1]); pk.y = pack_bf16(o[2], o[3]);
          pk.z = pack_bf16(o[4], o[5]); pk.w = pack_bf16(o[6], o[7]);
          *reinterpret_cast<uint4 *>(hr + j8) = pk;
          const bf16 *hb = reinterpret_cast<const bf16 *>(&pk);
#pragma unroll
          for (int j = 0; j < 8; j++) g.Ht[(long long)(nb + j8 + j) * g.ldht + m] = hb[j];
        }
      } else if (EPI == EPI_OUT) {
        float *cr = g.C + (long long)m * g.ldc + nb;
#pragma unroll
        for (int j = 0; j < CW; j++) cr[j] = v[j] + (nb + j < g.nvalid ? __ldg(g.bias + nb + j) : 0.f);
      } else {
#pragma unroll
        for (int j = 0; j < CW; j++)
          if (nb + j < g.nvalid)
            atomicAdd(g.ctrans ? g.C + (long long)(nb + j) * g.ldc + m : g.C + (long long)m * g.ldc + nb + j, v[j]);
      }
    }
  } else if (!ok && threadIdx.x == 0) {
    atomicExch(g.err, 1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(NCOL));
}

// error map: per tile the largest |s - v| / max(|v|, c_f) over points and flavours
__global__ void k_tile_err(SurrConst c, const double *xa, const double *qa, long long n, const float *s,
                           const double *v, unsigned int *tile_err_bits, unsigned int *tile_cnt) {
  long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  float z0, z1;
  point_z(c, xa[p], qa[p], z0, z1);
  if (!(z0 >= -1.f && z0 <= 1.f && z1 >= -1.f && z1 <= 1.f)) return;
  int tx = min(MAPN - 1, (int)((z0 + 1.f) * 0.5f * MAPN)), tq = min(MAPN - 1, (int)((z1 + 1.f) * 0.5f * MAPN));
  float e = 0.f;
  for (int f = 0; f < c.nf; f++) {
    double vv = v[p * c.nf + f];
    double d = fabs((double)s[p * c.nf + f] - vv) / fmax(fabs(vv), (double)c.scale[f]);
    e = fmaxf(e, (float)d);
  }
  if (isnan(e)) e = 1e30f;
  atomicMax(tile_err_bits + tq * MAPN + tx, __float_as_uint(e));  // e >= 0: bits order like values
  if (tile_cnt) atomicAdd(tile_cnt + tq * MAPN + tx, 1u);
}

// tile states: 0 the interpolator, 1 the network, 2 the residual target's
// base alone (its network term left out): the more accurate of 1 and 2 among
// those within the threshold
__global__ void k_make_mask(const unsigned int *tile_err_bits, const unsigned int *base_err_bits,
                            const unsigned int *tile_cnt, float thr, unsigned char *mask) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= MAPN * MAPN) return;
  const float en = __uint_as_float(tile_err_bits[t]);
  const float eb = base_err_bits ? __uint_as_float(base_err_bits[t]) : INFINITY;
  unsigned char m = 0;
  if (tile_cnt[t] > 0) {
    if (en <= thr && en <= eb) m = 1;
    else if (eb <= thr) m = 2;
    else if (en <= thr) m = 1;
  }
  mask[t] = m;
}

__global__ void k_gather(const double *x, const double *q2, const unsigned int *idx, unsigned int m, double *gx,
                         double *gq) {
  unsigned int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  gx[i] = x[idx[i]];
  gq[i] = q2[idx[i]];
}
__global__ void k_scatter(const double *src, const unsigned int *idx, unsigned int m, int nf, double *out) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)m * nf) return;
  long long r = i / nf;
  out[(long long)idx[r] * nf + (i % nf)] = src[i];
}

int cuda_err(cudaError_t e, const char *what) {
  if (e == cudaSuccess) return PDF_OK;
  return set_error(PDF_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

}  // namespace

struct pdf_surrogate {
  std::mutex mu;  // serialises the calls that use the scratch below (all but pdf_surrogate_eval)
  int nf, max_batch, device;
  Layout L;
  SurrConst c;
  float *params, *grads, *am, *av;  // device FP32
  float *scale_d;                   // device copy of c_f
  bf16 *wbf;                        // device BF16 copies
  // training scratch (max_batch rows)
  bf16 *h[5], *g[5];  // h0 [B][32], h1..h4 [B][128]; g1..g4 [B][128], g5 [B][16] at index 0..4 (g[l] for layer l)
  bf16 *ht[5], *gt[5];  // their transposes [columns][bt]
  bf16 *wt;             // transposed BF16 weights of layers 1..4 (wt_off)
  long long bt;         // row stride of the transposes (max_batch rounded up to 64)
  double *xb, *qb;      // the training step's batch
  TrainState *ts;       // the training call's step state
  cudaStream_t tstream; // training runs here (a capturable stream), ordered with the caller's by events
  cudaEvent_t tev[2];
  float *z[4], *y, *t;
  int last_n;  // points of the last loss/gradient pass (pdf_surrogate_trace reads its buffers)
  double *xfbuf, *loss;
  long long step;
  // error map and fallback
  unsigned char *mask;
  unsigned int *tile_bits, *base_bits, *tile_cnt, *nfb, *fb_idx;
  int *tc_err;  // set by the inference kernel when a tensor-core wait ran out
  double *fb_x, *fb_q, *fb_out;
  size_t fb_cap;
  // recorded after a fallback call's last use of fb_*: the next call's stream
  // waits on it, so a call on another stream cannot overwrite them early
  cudaEvent_t fb_done;
  bool fb_pending;
  bool has_map;
  std::vector<void *> blocks;
  template <typename T>
  int alloc(T **p, size_t count) {
    void *q = nullptr;
    if (cudaMalloc(&q, count * sizeof(T)) != cudaSuccess) return set_error(PDF_ERR_ALLOC, "surrogate: cudaMalloc");
    blocks.push_back(q);
    *p = static_cast<T *>(q);
    return PDF_OK;
  }
};

namespace {

template <int EPI, int NT>
void tg_launch(const TGemm &a, int ksplit, cudaStream_t st) {
  static const bool attr =  // once per instantiation (one device per process)
      cudaFuncSetAttribute(k_tgemm<EPI, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTgSmem) ==
      cudaSuccess;
  (void)attr;
  dim3 grid((unsigned)((a.M + 127) / 128), (unsigned)ksplit, (unsigned)((a.N + NT - 1) / NT));
  k_tgemm<EPI, NT><<<grid, 128, kTgSmem, st>>>(a);
}

// One forward + backward pass on a batch already in h[0] / ht[0] (features)
// and t (targets); gradients accumulate into s->grads (zeroed here).  Every
// product reads K-contiguous rows: forward H W^T; backward dH = G W (with the
// transposed weights), dW = G^T H over the batch (with the transposed
// gradients and activations the epilogues write).
int forward_backward(pdf_surrogate *s, int B, cudaStream_t st) {
  const Layout &L = s->L;
  const long long BT = s->bt;
  cudaMemsetAsync(s->grads, 0, L.total * sizeof(float), st);
  cudaMemsetAsync(s->loss, 0, sizeof(double), st);
  TGemm a{};
  a.err = s->tc_err;
  // forward: Z_l = H_l W_l^T + b_l, H_{l+1} = silu(Z_l)
  for (int l = 0; l < 4; l++) {
    const int K = l == 0 ? SIN : SW;
    a.A = s->h[l]; a.lda = K; a.B = s->wbf + wbf_off(l); a.ldb = K;
    a.M = B; a.N = SW; a.K = K; a.kchunk = K;
    a.bias = s->params + L.b[l];
    a.Z = s->z[l]; a.ldz = SW; a.H = s->h[l + 1]; a.ldh = SW; a.Ht = s->ht[l + 1]; a.ldht = BT;
    tg_launch<EPI_FWD_SILU, 64>(a, 1, st);
  }
  a.A = s->h[4]; a.lda = SW; a.B = s->wbf + wbf_off(4); a.ldb = SW;
  a.M = B; a.N = SOUT; a.K = SW; a.kchunk = SW;
  a.bias = s->params + L.b[4]; a.nvalid = s->nf;  // padded output columns carry no bias
  a.C = s->y; a.ldc = SOUT; a.ctrans = 0;
  tg_launch<EPI_OUT, SOUT>(a, 1, st);
  k_loss<<<(B * SOUT + 255) / 256, 256, 0, st>>>(s->y, s->t, B, s->nf, s->g[4], s->gt[4], BT, s->loss);
  // backward; the weight gradients sum over the batch in chunks of kTgBatch rows, added atomically
  const int ksplit = (B + kTgBatch - 1) / kTgBatch;
  for (int l = 4; l >= 0; l--) {
    const int in = l == 0 ? SIN : SW, out = l == 4 ? SOUT : SW, nout = l == 4 ? s->nf : SW;
    a.K = B; a.kchunk = kTgBatch; a.C = s->grads + L.w[l];
    if (l == 4) {  // dW_4^T[j][o] = sum_b H_4[b][j] G_4[b][o] (rows j: a 128-row tile)
      a.A = s->ht[4]; a.lda = BT; a.B = s->gt[4]; a.ldb = BT;
      a.M = SW; a.N = SOUT; a.nvalid = nout; a.ldc = SW; a.ctrans = 1;
      tg_launch<EPI_ATOMIC, SOUT>(a, ksplit, st);
    } else {       // dW_l[o][j] = sum_b G_l[b][o] H_l[b][j]
      a.A = s->gt[l]; a.lda = BT; a.B = s->ht[l]; a.ldb = BT;
      a.M = SW; a.N = in; a.nvalid = in; a.ldc = in; a.ctrans = 0;
      if (l == 0) tg_launch<EPI_ATOMIC, SIN>(a, ksplit, st);
      else tg_launch<EPI_ATOMIC, 64>(a, ksplit, st);
    }
    k_colsum<<<(B + kColRows - 1) / kColRows, 128, 0, st>>>(s->g[l], B, out, nout, s->grads + L.b[l]);
    if (l > 0) {  // dH_l[b][j] = sum_o G_l[b][o] W_l[o][j] -> G_{l-1} = dH silu'(Z_{l-1})
      a.A = s->g[l]; a.lda = out; a.B = s->wt + wt_off(l); a.ldb = out;
      a.M = B; a.N = in; a.K = out; a.kchunk = out;
      a.Z = s->z[l - 1]; a.ldz = SW; a.H = s->g[l - 1]; a.ldh = SW; a.Ht = s->gt[l - 1]; a.ldht = BT;
      tg_launch<EPI_BWD_SILU, 64>(a, 1, st);
    }
  }
  return check_launch("surrogate forward/backward");
}

void cast_weights(pdf_surrogate *s, cudaStream_t st, TrainState *ts = nullptr) {
  CastArgs a;
  a.ts = ts;
  a.p = s->params;
  a.w = s->wbf;
  a.wt = s->wt;
  for (int l = 0; l < 5; l++) { a.woff[l] = s->L.w[l]; a.boff[l] = s->L.b[l]; }
  a.nf = s->nf;
  k_cast<<<(unsigned)((kWbfTotal + kWtTotal + 255) / 256), 256, 0, st>>>(a);
}

int features_targets(pdf_surrogate *s, const pdf_grid *grid, const double *x, const double *q2, int B,
                     const double *xf_given, cudaStream_t st) {
  k_features<<<(B * SIN + 255) / 256, 256, 0, st>>>(s->c, x, q2, B, s->h[0], s->ht[0], s->bt);
  const double *xf = xf_given;
  if (!xf) {
    int rc = launch_all_f64(grid, x, q2, B, s->xfbuf, nullptr, st);
    if (rc) return rc;
    xf = s->xfbuf;
  }
  k_targets<<<(B * SOUT + 255) / 256, 256, 0, st>>>(s->c, x, q2, xf, B, s->t);
  return check_launch("surrogate features/targets");
}

}  // namespace

using namespace pdfgb;

// Fills a new surrogate (its pointers null); on failure the caller frees it.
static int create_body(pdf_surrogate *s, const pdf_grid *grid, const float *params, const float *freq,
                       int max_batch, int target) {
  const int nf = grid->v.nf;
  s->nf = nf;
  s->max_batch = max_batch;
  cudaGetDevice(&s->device);
  s->L.set(nf);
  // constants: input normalisation from the grid's knot range, flavour scales
  // c_f = 1e-5 max |xf_f| over the knots
  const GridView &v = grid->v;
  std::vector<double> vals((size_t)v.nrows * v.nx * v.nf);
  int rc = cuda_err(cudaMemcpy(vals.data(), v.vals, vals.size() * sizeof(double), cudaMemcpyDeviceToHost),
                    "pdf_surrogate_create");
  if (rc) return rc;
  for (int f = 0; f < SOUT; f++) s->c.scale[f] = 1.f;
  for (int f = 0; f < nf; f++) {
    double m = 0.0;
    for (size_t k = f; k < vals.size(); k += nf) m = fmax(m, fabs(vals[k]));
    s->c.scale[f] = (float)(1e-5 * (m > 0.0 ? m : 1.0));
  }
  double lxlo = log(v.x0), lxhi = log(v.xlast), lqlo = log(v.q2min), lqhi = log(v.q2max);
  // envelope table: E_f(x_i) = max over Q rows of |xf_f(x_i, Q)| (at least c_f),
  // ln E_f linear in ln x between knots, sampled at ENVN + 1 equal steps
  std::vector<double> xk(v.nx);
  rc = cuda_err(cudaMemcpy(xk.data(), v.xk, v.nx * sizeof(double), cudaMemcpyDeviceToHost), "pdf_surrogate_create");
  if (rc) return rc;
  std::vector<float> envt((size_t)(ENVN + 1) * SOUT, 0.f);
  {
    std::vector<double> lx(v.nx), le(v.nx);
    for (int i = 0; i < v.nx; i++) lx[i] = log(xk[i]);
    for (int f = 0; f < nf; f++) {
      for (int i = 0; i < v.nx; i++) {
        double m = 0.0;
        for (int j = 0; j < v.nrows; j++) m = fmax(m, fabs(vals[((size_t)j * v.nx + i) * nf + f]));
        le[i] = log(fmax(m, (double)s->c.scale[f]));
      }
      for (int k = 0; k <= ENVN; k++) {
        const double l = lxlo + (lxhi - lxlo) * k / ENVN;
        int i = 0;
        while (i + 2 < v.nx && lx[i + 1] <= l) i++;
        const double t = fmin(fmax((l - lx[i]) / (lx[i + 1] - lx[i]), 0.0), 1.0);
        envt[(size_t)k * SOUT + f] = (float)(le[i] + t * (le[i + 1] - le[i]));
      }
    }
  }
  s->c.target = target;
  s->c.baset = nullptr;
  s->c.lx_lo = (float)lxlo; s->c.inv_lx = (float)(1.0 / (lxhi - lxlo));
  s->c.lq_lo = (float)lqlo; s->c.inv_lq = (float)(1.0 / (lqhi - lqlo));
  for (int j = 0; j < SNQ; j++) { s->c.freq[j][0] = freq[2 * j]; s->c.freq[j][1] = freq[2 * j + 1]; }
  s->c.nf = nf;
  const size_t P = s->L.total, B = (size_t)max_batch;
  rc = s->alloc(&s->params, P);
  if (!rc) rc = s->alloc(&s->grads, P);
  if (!rc) rc = s->alloc(&s->am, P);
  if (!rc) rc = s->alloc(&s->av, P);
  if (!rc) rc = s->alloc(&s->scale_d, SOUT);
  float *envt_d = nullptr;
  if (!rc) rc = s->alloc(&envt_d, envt.size());
  if (!rc) rc = s->alloc(&s->wbf, kWbfTotal);
  if (!rc) rc = s->alloc(&s->h[0], B * SIN);
  for (int l = 1; l < 5 && !rc; l++) rc = s->alloc(&s->h[l], B * SW);
  for (int l = 0; l < 4 && !rc; l++) rc = s->alloc(&s->g[l], B * SW);
  if (!rc) rc = s->alloc(&s->g[4], B * SOUT);
  for (int l = 0; l < 4 && !rc; l++) rc = s->alloc(&s->z[l], B * SW);
  s->bt = (long long)((B + 63) / 64 * 64);
  if (!rc) rc = s->alloc(&s->ht[0], (size_t)SIN * s->bt);
  for (int l = 1; l < 5 && !rc; l++) rc = s->alloc(&s->ht[l], (size_t)SW * s->bt);
  for (int l = 0; l < 4 && !rc; l++) rc = s->alloc(&s->gt[l], (size_t)SW * s->bt);
  if (!rc) rc = s->alloc(&s->gt[4], (size_t)SOUT * s->bt);
  if (!rc) rc = s->alloc(&s->wt, kWtTotal);
  if (!rc) rc = s->alloc(&s->xb, (size_t)B);
  if (!rc) rc = s->alloc(&s->qb, (size_t)B);
  if (!rc) rc = s->alloc(&s->ts, 1);
  if (!rc && cudaStreamCreateWithFlags(&s->tstream, cudaStreamNonBlocking) != cudaSuccess)
    rc = set_error(PDF_ERR_CUDA, "pdf_surrogate_create: training stream");
  for (int k = 0; k < 2 && !rc; k++)
    if (cudaEventCreateWithFlags(&s->tev[k], cudaEventDisableTiming) != cudaSuccess)
      rc = set_error(PDF_ERR_CUDA, "pdf_surrogate_create: training events");
  if (!rc && cudaEventCreateWithFlags(&s->fb_done, cudaEventDisableTiming) != cudaSuccess)
    rc = set_error(PDF_ERR_CUDA, "pdf_surrogate_create: fallback event");
  if (!rc) rc = s->alloc(&s->y, B * SOUT);
  if (!rc) rc = s->alloc(&s->t, B * SOUT);
  if (!rc) rc = s->alloc(&s->xfbuf, B * nf);
  if (!rc) rc = s->alloc(&s->loss, 1);
  if (!rc) rc = s->alloc(&s->mask, MAPN * MAPN);
  if (!rc) rc = s->alloc(&s->tile_bits, MAPN * MAPN);
  if (!rc) rc = s->alloc(&s->base_bits, MAPN * MAPN);
  if (!rc) rc = s->alloc(&s->tile_cnt, MAPN * MAPN);
  if (!rc) rc = s->alloc(&s->nfb, 1);
  if (!rc) rc = s->alloc(&s->tc_err, 1);
  if (rc) return rc;
  const char *what = "pdf_surrogate_create";
  rc = cuda_err(cudaMemcpy(s->params, params, P * sizeof(float), cudaMemcpyHostToDevice), what);
  if (!rc) rc = cuda_err(cudaMemcpy(s->scale_d, s->c.scale, SOUT * sizeof(float), cudaMemcpyHostToDevice), what);
  if (!rc) rc = cuda_err(cudaMemcpy(envt_d, envt.data(), envt.size() * sizeof(float), cudaMemcpyHostToDevice), what);
  if (!rc) rc = cuda_err(cudaMemset(s->am, 0, P * sizeof(float)), what);
  if (!rc) rc = cuda_err(cudaMemset(s->av, 0, P * sizeof(float)), what);
  if (!rc) rc = cuda_err(cudaMemset(s->mask, 0, MAPN * MAPN), what);
  if (!rc) rc = cuda_err(cudaMemset(s->tc_err, 0, sizeof(int)), what);
  if (rc) return rc;
  s->c.envt = envt_d;
  if (target == PDF_SURR_RESIDUAL) {
    // base table: the FP64 interpolator at the (BASEN + 1)^2 nodes of (z0, z1), rounded to FP32
    const size_t nn = (size_t)(BASEN + 1) * (BASEN + 1);
    std::vector<double> bx(nn), bq(nn);
    for (int i = 0; i <= BASEN; i++)
      for (int j = 0; j <= BASEN; j++) {
        bx[(size_t)i * (BASEN + 1) + j] = i == BASEN ? v.xlast : exp(lxlo + (lxhi - lxlo) * i / BASEN);
        bq[(size_t)i * (BASEN + 1) + j] = j == BASEN ? v.q2max : exp(lqlo + (lqhi - lqlo) * j / BASEN);
      }
    bx[0] = v.x0;
    double *dx = nullptr, *dq = nullptr, *dv = nullptr;
    float *bt = nullptr;
    rc = s->alloc(&bt, nn * SOUT);
    if (!rc) rc = cuda_err(cudaMalloc(&dx, nn * sizeof(double)), what);
    if (!rc) rc = cuda_err(cudaMalloc(&dq, nn * sizeof(double)), what);
    if (!rc) rc = cuda_err(cudaMalloc(&dv, nn * nf * sizeof(double)), what);
    for (size_t k = 0; k < nn; k++) {  // the nodes on the low edges are the knots themselves
      if (k % (BASEN + 1) == 0) bq[k] = v.q2min;
      if (k < (size_t)(BASEN + 1)) bx[k] = v.x0;
    }
    if (!rc) rc = cuda_err(cudaMemcpy(dx, bx.data(), nn * sizeof(double), cudaMemcpyHostToDevice), what);
    if (!rc) rc = cuda_err(cudaMemcpy(dq, bq.data(), nn * sizeof(double), cudaMemcpyHostToDevice), what);
    if (!rc) rc = launch_all_f64(grid, dx, dq, (long long)nn, dv, nullptr, 0);
    std::vector<double> hv(rc ? 0 : nn * nf);
    if (!rc) rc = cuda_err(cudaMemcpy(hv.data(), dv, nn * nf * sizeof(double), cudaMemcpyDeviceToHost), what);
    if (dx) cudaFree(dx);
    if (dq) cudaFree(dq);
    if (dv) cudaFree(dv);
    if (rc) return rc;
    std::vector<float> ht(nn * SOUT, 0.f);
    for (size_t k = 0; k < nn; k++)
      for (int f = 0; f < nf; f++) ht[k * SOUT + f] = (float)hv[k * nf + f];
    rc = cuda_err(cudaMemcpy(bt, ht.data(), ht.size() * sizeof(float), cudaMemcpyHostToDevice), what);
    if (rc) return rc;
    s->c.baset = bt;
  }
  cast_weights(s, 0);
  return cuda_err(cudaDeviceSynchronize(), what);
}

extern "C" int pdf_surrogate_create_ex(const pdf_grid *grid, const float *params, const float *freq, int max_batch,
                                       int target, pdf_surrogate **out) {
  if (!grid || !params || !freq || !out) return set_error(PDF_ERR_NULL, "pdf_surrogate_create: NULL argument");
  *out = nullptr;
  if (target != PDF_SURR_ASINH && target != PDF_SURR_ENVELOPE && target != PDF_SURR_RESIDUAL)
    return set_error(PDF_ERR_ARG, "pdf_surrogate_create: unknown target %d", target);
  if (grid->v.nf > SOUT) return set_error(PDF_ERR_ARG, "pdf_surrogate_create: at most %d flavours", SOUT);
  if (max_batch < 16 || max_batch > (1 << 22))
    return set_error(PDF_ERR_ARG, "pdf_surrogate_create: max_batch %d outside [16, 4M]", max_batch);
  pdf_surrogate *s = new (std::nothrow) pdf_surrogate();
  if (!s) return set_error(PDF_ERR_ALLOC, "pdf_surrogate_create: host allocation");
  const int rc = guarded("pdf_surrogate_create",
                         [&] { return create_body(s, grid, params, freq, max_batch, target); });
  if (rc) {
    pdf_surrogate_free(s);
    return rc;
  }
  *out = s;
  return PDF_OK;
}

extern "C" int pdf_surrogate_create(const pdf_grid *grid, const float *params, const float *freq, int max_batch,
                                    pdf_surrogate **out) {
  return pdf_surrogate_create_ex(grid, params, freq, max_batch, PDF_SURR_ASINH, out);
}

extern "C" int pdf_surrogate_free(pdf_surrogate *s) {
  if (!s) return PDF_OK;
  if (s->tstream) {
    cudaStreamSynchronize(s->tstream);
    cudaStreamDestroy(s->tstream);
  }
  for (cudaEvent_t e : s->tev)
    if (e) cudaEventDestroy(e);
  if (s->fb_done) {
    cudaEventSynchronize(s->fb_done);
    cudaEventDestroy(s->fb_done);
  }
  for (void *p : {(void *)s->fb_idx, (void *)s->fb_x, (void *)s->fb_q, (void *)s->fb_out})
    if (p) cudaFree(p);
  for (void *p : s->blocks) cudaFree(p);
  delete s;
  return PDF_OK;
}

extern "C" int pdf_surrogate_nparams(const pdf_surrogate *s, size_t *n) {
  if (!s || !n) return set_error(PDF_ERR_NULL, "pdf_surrogate_nparams: NULL argument");
  *n = s->L.total;
  return PDF_OK;
}

extern "C" int pdf_surrogate_get_params(const pdf_surrogate *s, float *params) {
  if (!s || !params) return set_error(PDF_ERR_NULL, "pdf_surrogate_get_params: NULL argument");
  return cuda_err(cudaMemcpy(params, s->params, s->L.total * sizeof(float), cudaMemcpyDeviceToHost),
                  "pdf_surrogate_get_params");
}

extern "C" int pdf_surrogate_set_params(pdf_surrogate *s, const float *params) {
  if (!s || !params) return set_error(PDF_ERR_NULL, "pdf_surrogate_set_params: NULL argument");
  std::lock_guard<std::mutex> lock(s->mu);
  int rc = cuda_err(cudaMemcpy(s->params, params, s->L.total * sizeof(float), cudaMemcpyHostToDevice),
                    "pdf_surrogate_set_params");
  if (rc) return rc;
  cast_weights(s, 0);
  s->has_map = false;
  return cuda_err(cudaDeviceSynchronize(), "pdf_surrogate_set_params");
}

static int check_tc(const pdf_surrogate *s, const char *what);

extern "C" int pdf_surrogate_loss_grad(pdf_surrogate *s, const double *x, const double *q2, const double *xf,
                                       size_t n, double *loss, float *grad) {
  if (!s || !x || !q2 || !xf || !loss || !grad) return set_error(PDF_ERR_NULL, "pdf_surrogate_loss_grad: NULL argument");
  if (n < 1 || n > (size_t)s->max_batch)
    return set_error(PDF_ERR_ARG, "pdf_surrogate_loss_grad: n = %zu outside [1, %d]", n, s->max_batch);
  std::lock_guard<std::mutex> lock(s->mu);
  int rc = features_targets(s, nullptr, x, q2, (int)n, xf, 0);
  if (!rc) rc = forward_backward(s, (int)n, 0);
  if (rc) return rc;
  s->last_n = (int)n;
  double sum = 0.0;
  rc = cuda_err(cudaMemcpy(&sum, s->loss, sizeof(double), cudaMemcpyDeviceToHost), "pdf_surrogate_loss_grad");
  if (!rc) rc = cuda_err(cudaMemcpy(grad, s->grads, s->L.total * sizeof(float), cudaMemcpyDeviceToHost),
                         "pdf_surrogate_loss_grad");
  if (!rc) rc = check_tc(s, "pdf_surrogate_loss_grad");
  *loss = sum / ((double)n * s->nf);
  return rc;
}

// bfloat16 [rows][cols] with row stride ld -> FP32 [rows][cols]
__global__ void k_bf16_rows(const bf16 *a, int rows, int cols, int ld, float *out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= rows * cols) return;
  out[i] = __bfloat162float(a[(size_t)(i / cols) * ld + i % cols]);
}

extern "C" int pdf_surrogate_trace(pdf_surrogate *s, int what, int layer, float *out) {
  if (!s || !out) return set_error(PDF_ERR_NULL, "pdf_surrogate_trace: NULL argument");
  std::lock_guard<std::mutex> lock(s->mu);
  const int n = s->last_n;
  if (n < 1) return set_error(PDF_ERR_ARG, "pdf_surrogate_trace: no loss/gradient pass yet");
  // the pass may have run on any stream: wait for the device
  if (int rc = cuda_err(cudaDeviceSynchronize(), "pdf_surrogate_trace")) return rc;
  const int cols_h = layer == 0 ? SIN : SW, cols_g = layer == 4 ? SOUT : SW;
  const float *src = nullptr;
  const bf16 *srcb = nullptr;
  int cols = 0, ld = 0;
  if (what == 0 && layer >= 0 && layer <= 4) { srcb = s->h[layer]; cols = ld = cols_h; }
  else if (what == 1 && layer >= 0 && layer <= 3) { src = s->z[layer]; cols = ld = SW; }
  else if (what == 2 && layer >= 0 && layer <= 4) { srcb = s->g[layer]; cols = ld = cols_g; }
  else if (what == 3 && layer == 0) { src = s->y; cols = ld = SOUT; }
  else if (what == 4 && layer == 0) { src = s->t; cols = ld = SOUT; }
  else return set_error(PDF_ERR_ARG, "pdf_surrogate_trace: no buffer (what %d, layer %d)", what, layer);
  const size_t bytes = (size_t)n * cols * sizeof(float);
  int rc = PDF_OK;
  if (src) {
    rc = cuda_err(cudaMemcpy(out, src, bytes, cudaMemcpyDeviceToHost), "pdf_surrogate_trace");
  } else {
    float *tmp = nullptr;
    rc = cuda_err(cudaMalloc(&tmp, bytes), "pdf_surrogate_trace");
    if (!rc) {
      k_bf16_rows<<<(unsigned)(((size_t)n * cols + 255) / 256), 256>>>(srcb, n, cols, ld, tmp);
      rc = cuda_err(cudaMemcpy(out, tmp, bytes, cudaMemcpyDeviceToHost), "pdf_surrogate_trace");
      cudaFree(tmp);
    }
  }
  return rc;
}

extern "C" int pdf_surrogate_train(pdf_surrogate *s, const pdf_grid *grid, const double *x, const double *q2,
                                   size_t n, const pdf_train_config *cfg, double *final_loss, cudaStream_t st) {
  if (!s || !grid || !x || !q2 || !cfg) return set_error(PDF_ERR_NULL, "pdf_surrogate_train: NULL argument");
  const int B = cfg->batch;
  if (B < 16 || B > s->max_batch || (size_t)B > n)
    return set_error(PDF_ERR_ARG, "pdf_surrogate_train: batch %d outside [16, min(max_batch, n)]", B);
  if (grid->v.nf != s->nf) return set_error(PDF_ERR_ARG, "pdf_surrogate_train: grid flavours differ");
  if (cfg->steps < 1) return set_error(PDF_ERR_ARG, "pdf_surrogate_train: steps must be >= 1");
  std::lock_guard<std::mutex> lock(s->mu);
  s->last_n = 0;  // training reuses the buffers a trace would read
  const long long nb = (long long)(n / (size_t)B);  // whole batches per pass
  cudaStream_t ts = s->tstream;
  // one training step; everything that changes from step to step (the batch,
  // the learning rate, Adam's step count) is read from the device state, so
  // the same enqueued work serves every step
  auto step = [&]() -> int {
    k_batch<<<(B + 255) / 256, 256, 0, ts>>>(x, q2, nb, B, s->ts, s->xb, s->qb);
    int rc = features_targets(s, grid, s->xb, s->qb, B, nullptr, ts);
    if (!rc) rc = forward_backward(s, B, ts);
    if (rc) return rc;
    AdamArgs a{s->params, s->grads, s->am, s->av, s->L.total, cfg->lr, cfg->lr_min, 0.9f, 0.999f, 1e-8f,
               cfg->warmup, cfg->steps, s->ts};
    k_adam<<<(unsigned)((s->L.total + 255) / 256), 256, 0, ts>>>(a);
    cast_weights(s, ts, s->ts);
    return check_launch("pdf_surrogate_train");
  };
  int rc = cuda_err(cudaEventRecord(s->tev[0], st), "pdf_surrogate_train");  // after the caller's work
  if (!rc) rc = cuda_err(cudaStreamWaitEvent(ts, s->tev[0], 0), "pdf_surrogate_train");
  if (rc) return rc;
  k_train_state<<<1, 1, 0, ts>>>(s->ts, s->step);
  rc = step();  // the first step directly (it also settles every kernel's launch attributes)
  if (!rc && cfg->steps > 1) {
    // the rest: one step captured as a CUDA graph and replayed (a step is ~26
    // small dependent launches; replaying the graph spares their launch cost)
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    rc = cuda_err(cudaStreamBeginCapture(ts, cudaStreamCaptureModeThreadLocal), "pdf_surrogate_train capture");
    if (!rc) {
      const int rs = step();
      const cudaError_t e = cudaStreamEndCapture(ts, &graph);
      rc = rs ? rs : cuda_err(e, "pdf_surrogate_train capture");
    }
    if (!rc) rc = cuda_err(cudaGraphInstantiate(&exec, graph, 0), "pdf_surrogate_train graph");
    for (int it = 1; it < cfg->steps && !rc; it++) rc = cuda_err(cudaGraphLaunch(exec, ts), "pdf_surrogate_train");
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
  }
  double last = 0.0;
  if (!rc) rc = cuda_err(cudaMemcpyAsync(&last, s->loss, sizeof(double), cudaMemcpyDeviceToHost, ts), "train");
  if (!rc) rc = cuda_err(cudaStreamSynchronize(ts), "pdf_surrogate_train");
  if (!rc) rc = check_tc(s, "pdf_surrogate_train");
  cudaEventRecord(s->tev[1], ts);  // the caller's later work comes after training
  cudaStreamWaitEvent(st, s->tev[1], 0);
  if (rc) return rc;
  s->step += cfg->steps;
  s->has_map = false;
  if (final_loss) *final_loss = last / ((double)B * s->nf);
  return PDF_OK;
}

// After a synchronisation: did an inference kernel give up on a tensor-core wait?
static int check_tc(const pdf_surrogate *s, const char *what) {
  int e = 0;
  int rc = cuda_err(cudaMemcpy(&e, s->tc_err, sizeof(int), cudaMemcpyDeviceToHost), what);
  if (!rc && e) {
    cudaMemset(s->tc_err, 0, sizeof(int));  // reported once
    rc = set_error(PDF_ERR_CUDA, "%s: a tensor-core wait in the inference kernel ran out", what);
  }
  return rc;
}

static int launch_infer(const pdf_surrogate *s, const double *x, const double *q2, size_t n, float *outf,
                        double *outd, const unsigned char *mask, unsigned int *nfb, unsigned int *idx,
                        cudaStream_t st) {
  static const bool attr =  // once (one device per process)
      cudaFuncSetAttribute(k_infer, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmem) == cudaSuccess;
  (void)attr;
  static const int sms = [] {
    int d = 0, m = 0;
    cudaGetDevice(&d);
    cudaDeviceGetAttribute(&m, cudaDevAttrMultiProcessorCount, d);
    return m > 0 ? m : 1;
  }();
  long long tiles = ((long long)n + 127) / 128;
  long long blocks = (tiles + TG - 1) / TG;
  if (blocks > sms) blocks = sms;
  k_infer<<<(unsigned)blocks, kTcThreads, kTcSmem, st>>>(s->c, s->wbf, s->params, s->L, x, q2, (long long)n, outf,
                                                          outd, mask, nfb, idx, s->tc_err);
  return check_launch("surrogate inference");
}

extern "C" int pdf_surrogate_eval(const pdf_surrogate *s, const double *x, const double *q2, size_t n, float *out,
                                  cudaStream_t st) {
  if (!s) return set_error(PDF_ERR_NULL, "pdf_surrogate_eval: surrogate is NULL");
  if (n > 0 && (!x || !q2 || !out)) return set_error(PDF_ERR_NULL, "pdf_surrogate_eval: NULL array");
  if (n == 0) return PDF_OK;
  return launch_infer(s, x, q2, n, out, nullptr, nullptr, nullptr, nullptr, st);
}

static int error_map_body(pdf_surrogate *s, const pdf_grid *grid, const double *x, const double *q2, size_t n,
                          double threshold, double *stats) {
  std::lock_guard<std::mutex> lock(s->mu);
  const bool res = s->c.target == PDF_SURR_RESIDUAL;
  // host copies first, so that nothing below can throw while device scratch is held
  std::vector<unsigned int> bits(MAPN * MAPN), bbits(MAPN * MAPN), cnt(MAPN * MAPN);
  std::vector<unsigned char> m(MAPN * MAPN);
  std::vector<float> errs;
  errs.reserve(MAPN * MAPN);
  float *sv = nullptr, *bv = nullptr;
  double *iv = nullptr;
  int rc = cuda_err(cudaMalloc(&sv, n * s->nf * sizeof(float)), "error map");
  if (!rc) rc = cuda_err(cudaMalloc(&iv, n * s->nf * sizeof(double)), "error map");
  if (!rc && res) rc = cuda_err(cudaMalloc(&bv, n * s->nf * sizeof(float)), "error map");
  if (!rc) rc = launch_infer(s, x, q2, n, sv, nullptr, nullptr, nullptr, nullptr, 0);
  if (!rc) rc = launch_all_f64(grid, x, q2, (long long)n, iv, nullptr, 0);
  if (!rc) {
    cudaMemset(s->tile_bits, 0, MAPN * MAPN * sizeof(unsigned int));
    cudaMemset(s->base_bits, 0, MAPN * MAPN * sizeof(unsigned int));
    cudaMemset(s->tile_cnt, 0, MAPN * MAPN * sizeof(unsigned int));
    const unsigned blocks = (unsigned)((n + 255) / 256);
    k_tile_err<<<blocks, 256>>>(s->c, x, q2, (long long)n, sv, iv, s->tile_bits, s->tile_cnt);
    if (res) {  // the base alone on the same points (counts taken once)
      const long long items = (long long)n * s->nf;
      k_base<<<(unsigned)((items + 255) / 256), 256>>>(s->c, x, q2, (long long)n, bv, nullptr);
      k_tile_err<<<blocks, 256>>>(s->c, x, q2, (long long)n, bv, iv, s->base_bits, nullptr);
    }
    k_make_mask<<<(MAPN * MAPN + 255) / 256, 256>>>(s->tile_bits, res ? s->base_bits : nullptr, s->tile_cnt,
                                                    (float)threshold, s->mask);
    rc = check_launch("error map");
  }
  if (!rc) rc = cuda_err(cudaMemcpy(bits.data(), s->tile_bits, bits.size() * 4, cudaMemcpyDeviceToHost), "error map");
  if (!rc) rc = cuda_err(cudaMemcpy(bbits.data(), s->base_bits, bbits.size() * 4, cudaMemcpyDeviceToHost), "error map");
  if (!rc) rc = cuda_err(cudaMemcpy(cnt.data(), s->tile_cnt, cnt.size() * 4, cudaMemcpyDeviceToHost), "error map");
  if (!rc) rc = cuda_err(cudaMemcpy(m.data(), s->mask, m.size(), cudaMemcpyDeviceToHost), "error map");
  cudaFree(sv);
  cudaFree(iv);
  if (bv) cudaFree(bv);
  if (!rc) rc = check_tc(s, "pdf_surrogate_build_error_map");
  if (rc) return rc;
  // stats: [tiles accepted, tiles with samples, largest error on sampled tiles, median tile error];
  // a tile's error is that of the way it is served (of the better way, if neither passes)
  int ok = 0, sampled = 0;
  float worst = 0.f;
  for (size_t t = 0; t < bits.size(); t++) {
    ok += m[t] != 0;
    if (cnt[t] > 0) {
      sampled++;
      float e, eb;
      std::memcpy(&e, &bits[t], 4);
      std::memcpy(&eb, &bbits[t], 4);
      if (res && (m[t] == 2 || (m[t] == 0 && eb < e))) e = eb;
      worst = fmaxf(worst, e);
      errs.push_back(e);
    }
  }
  if (stats) {
    stats[0] = ok;
    stats[1] = sampled;
    stats[2] = worst;
    if (!errs.empty()) {
      std::nth_element(errs.begin(), errs.begin() + errs.size() / 2, errs.end());
      stats[3] = errs[errs.size() / 2];
    } else {
      stats[3] = 0.0;
    }
  }
  s->has_map = true;
  return PDF_OK;
}

extern "C" int pdf_surrogate_build_error_map(pdf_surrogate *s, const pdf_grid *grid, const double *x,
                                             const double *q2, size_t n, double threshold, double *stats) {
  if (!s || !grid || !x || !q2) return set_error(PDF_ERR_NULL, "pdf_surrogate_build_error_map: NULL argument");
  if (n == 0) return set_error(PDF_ERR_ARG, "pdf_surrogate_build_error_map: no validation points");
  if (grid->v.nf != s->nf) return set_error(PDF_ERR_ARG, "pdf_surrogate_build_error_map: grid flavours differ");
  return guarded("pdf_surrogate_build_error_map",
                 [&] { return error_map_body(s, grid, x, q2, n, threshold, stats); });
}

extern "C" int pdf_surrogate_map(pdf_surrogate *s, unsigned char *states) {
  if (!s || !states) return set_error(PDF_ERR_NULL, "pdf_surrogate_map: NULL argument");
  std::lock_guard<std::mutex> lock(s->mu);
  if (!s->has_map) return set_error(PDF_ERR_ARG, "pdf_surrogate_map: build the error map first");
  return cuda_err(cudaMemcpy(states, s->mask, MAPN * MAPN, cudaMemcpyDeviceToHost), "pdf_surrogate_map");
}

extern "C" int pdf_surrogate_eval_fallback(pdf_surrogate *s, const pdf_grid *grid, const double *x,
                                           const double *q2, size_t n, double *out, unsigned long long *n_fallback,
                                           cudaStream_t st) {
  if (!s || !grid) return set_error(PDF_ERR_NULL, "pdf_surrogate_eval_fallback: NULL argument");
  if (n > 0 && (!x || !q2 || !out)) return set_error(PDF_ERR_NULL, "pdf_surrogate_eval_fallback: NULL array");
  if (grid->v.nf != s->nf) return set_error(PDF_ERR_ARG, "pdf_surrogate_eval_fallback: grid flavours differ");
  if (!s->has_map) return set_error(PDF_ERR_ARG, "pdf_surrogate_eval_fallback: build the error map first");
  if (n > 0xFFFFFFFFull) return set_error(PDF_ERR_ARG, "pdf_surrogate_eval_fallback: n too large");
  if (n == 0) { if (n_fallback) *n_fallback = 0; return PDF_OK; }
  std::lock_guard<std::mutex> lock(s->mu);
  // the previous call (perhaps on another stream) may still read fb_* (its
  // gather, fallback evaluation and scatter run after its count is known)
  if (s->fb_pending && cudaStreamWaitEvent(st, s->fb_done, 0) != cudaSuccess)
    return cuda_err(cudaGetLastError(), "pdf_surrogate_eval_fallback: ordering after the previous call");
  if (n > s->fb_cap) {
    for (void *p : {(void *)s->fb_idx, (void *)s->fb_x, (void *)s->fb_q, (void *)s->fb_out}) if (p) cudaFree(p);
    s->fb_idx = nullptr; s->fb_x = s->fb_q = s->fb_out = nullptr; s->fb_cap = 0;
    int rc = cuda_err(cudaMalloc(&s->fb_idx, n * sizeof(unsigned int)), "fallback buffers");
    if (!rc) rc = cuda_err(cudaMalloc(&s->fb_x, n * sizeof(double)), "fallback buffers");
    if (!rc) rc = cuda_err(cudaMalloc(&s->fb_q, n * sizeof(double)), "fallback buffers");
    if (!rc) rc = cuda_err(cudaMalloc(&s->fb_out, n * s->nf * sizeof(double)), "fallback buffers");
    if (rc) return rc;
    s->fb_cap = n;
  }
  cudaMemsetAsync(s->nfb, 0, sizeof(unsigned int), st);
  int rc = launch_infer(s, x, q2, n, nullptr, out, s->mask, s->nfb, s->fb_idx, st);
  if (rc) return rc;
  unsigned int m = 0;
  rc = cuda_err(cudaMemcpyAsync(&m, s->nfb, sizeof(m), cudaMemcpyDeviceToHost, st), "fallback count");
  if (!rc) rc = cuda_err(cudaStreamSynchronize(st), "fallback count");
  if (!rc) rc = check_tc(s, "pdf_surrogate_eval_fallback");
  if (rc) return rc;
  if (m > 0) {
    k_gather<<<(m + 255) / 256, 256, 0, st>>>(x, q2, s->fb_idx, m, s->fb_x, s->fb_q);
    rc = launch_all_f64(grid, s->fb_x, s->fb_q, (long long)m, s->fb_out, nullptr, st);
    if (!rc)
      k_scatter<<<(unsigned)(((long long)m * s->nf + 255) / 256), 256, 0, st>>>(s->fb_out, s->fb_idx, m, s->nf,
                                                                                out);
  }
  s->fb_pending = cudaEventRecord(s->fb_done, st) == cudaSuccess;
  if (rc) return rc;
  if (n_fallback) *n_fallback = m;
  return check_launch("pdf_surrogate_eval_fallback");
}
