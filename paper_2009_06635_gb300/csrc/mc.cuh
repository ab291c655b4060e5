// mc.cuh -- counter-based event generation for the Monte Carlo integration
// (the PDF load of PDFFlow Sec. 4.1 inside a VegasFlow-style loop, Sec. 5).
//
// Event i draws u1 = U(z_{2i}), u2 = U(z_{2i+1}), z_k the k-th output of
// SplitMix64 (G. L. Steele, D. Lea, C. H. Flood, "Fast splittable
// pseudorandom number generators", OOPSLA 2014): the state after k + 1 steps
// is seed + (k + 1) * 0x9E3779B97F4A7C15, passed through the generator's
// 64-bit finaliser; U(z) = (z >> 11) * 2^-53 in [0, 1).  Then
// ln x_j = ln x_max + u_j (ln x_min - ln x_max), so x_j covers [x_min, x_max]
// with density 1 / (x_j (ln x_max - ln x_min)) (x_j capped at x_max against
// the rounding of exp).  A counter-based generator needs no state: any chunk
// of events can be generated anywhere, in any order.  The exponential is the
// table-driven one of tang.cuh (within 2 ulp, ~10 FP64 operations against
// ~25 for the device library's): the event kernels and the weights each
// regenerate the events, and on GB300 the FP64 pipe is the scarce one.
#pragma once

#include "tang.cuh"

namespace pdfgb {

struct McGen {
  unsigned long long seed;   // generator seed
  unsigned long long first;  // global index of the launch's first event
  double lxmin, lxmax;       // ln x_min, ln x_max
  double xmax;               // x_max (exp may round ln x_max's image above it)
  int on;                    // 1: generate x1, x2; 0: read them
  const double *et;          // tang.cuh's table 2^(k/256) (the grid's texptab)
  int cut;                   // 1: events with x1 x2 s below shat_min are not evaluated
  double shat_min;           // (their weight is zero: the integration never reads their rows)
  int near_only;             // 1: no evaluated event can need a continuation rule (no far launch)
  double *shat_out;          // non-null: x1 x2 s of every event of the launch, cut or not
};

__host__ __device__ inline unsigned long long splitmix64(unsigned long long seed, unsigned long long k) {
  unsigned long long z = seed + (k + 1) * 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

// x1, x2 of event i of the launch (global index gen.first + i).
__device__ __forceinline__ void mc_event(const McGen &gen, unsigned long long i, double &x1, double &x2) {
  const unsigned long long k = 2 * (gen.first + i);
  const double u1 = (double)(splitmix64(gen.seed, k) >> 11) * 0x1p-53;
  const double u2 = (double)(splitmix64(gen.seed, k + 1) >> 11) * 0x1p-53;
  const double span = gen.lxmin - gen.lxmax;
  x1 = fmin(texp(gen.lxmax + u1 * span, gen.et), gen.xmax);
  x2 = fmin(texp(gen.lxmax + u2 * span, gen.et), gen.xmax);
}

}  // namespace pdfgb
