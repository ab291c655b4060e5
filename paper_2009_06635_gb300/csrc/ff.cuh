// ff.cuh -- float-float arithmetic on the FP32 pipe (a value is hi + lo, two
// floats, ~48 bits of significand), shared by the FP64 evaluation and the
// adjoint: on GB300 the FP32 pipe issues 64 times as many operations as the
// FP64 pipe, so contractions that tolerate ~2^-46 relative rounding run here.
#pragma once

#include <cuda_runtime.h>

namespace pdfgb {

// Error-free product (FMA) and sum (TwoSum); the _rn intrinsics keep the
// compiler from contracting or reordering the error terms.
struct ff2 {
  float h, l;
};
// Exact float -> double on the integer pipe for normal floats and zeros (the
// FP64 pipe's conversion costs as much as an FMA on GB300); subnormals,
// infinities and NaN take the hardware conversion.
__device__ __forceinline__ double f2d(float f) {
  const unsigned b = __float_as_uint(f), a = b & 0x7FFFFFFFu;
  if (a - 0x00800000u < 0x7F000000u)  // biased exponent in [1, 254]
    return __hiloint2double((int)(((a >> 3) + 0x38000000u) | (b & 0x80000000u)), (int)(b << 29));
  if (a == 0u) return __hiloint2double((int)(b & 0x80000000u), 0);
  return (double)f;
}
// a double as hi + lo (the hi part back to double on the integer pipe)
__device__ __forceinline__ ff2 ff_of(double a) {
  float h = __double2float_rn(a);
  return {h, __double2float_rn(a - f2d(h))};
}
__device__ __forceinline__ ff2 ff_mul(ff2 a, ff2 b) {
  float p = __fmul_rn(a.h, b.h);
  float e = __fmaf_rn(a.h, b.h, -p);
  e = __fmaf_rn(a.h, b.l, __fmaf_rn(a.l, b.h, e));
  float h = __fadd_rn(p, e);
  return {h, __fsub_rn(e, __fsub_rn(h, p))};
}
__device__ __forceinline__ void ff_bernstein(double t, double s, ff2 *B) {
  const ff2 tf = ff_of(t), sf = ff_of(s), three = {3.f, 0.f};
  const ff2 t2 = ff_mul(tf, tf), s2 = ff_mul(sf, sf);
  B[0] = ff_mul(s2, sf);
  B[1] = ff_mul(three, ff_mul(tf, s2));
  B[2] = ff_mul(three, ff_mul(t2, sf));
  B[3] = ff_mul(t2, tf);
}
// -a of a packed pair (operands of the f32x2 intrinsics __fadd2_rn, __ffma2_rn)
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
// s += w b, s an unnormalised pair (sum, gathered rounding errors): exact
// product, TwoSum of the high parts, the cross terms and errors in s_l
__device__ __forceinline__ void ff_acc(float &sh, float &sl, ff2 w, float bh, float bl) {
  const float ph = __fmul_rn(w.h, bh);
  float pe = __fmaf_rn(w.h, bh, -ph);
  pe = __fmaf_rn(w.h, bl, __fmaf_rn(w.l, bh, pe));
  const float t = __fadd_rn(sh, ph);
  const float bp = __fsub_rn(t, sh);
  const float err = __fadd_rn(__fsub_rn(sh, __fsub_rn(t, bp)), __fsub_rn(ph, bp));
  sh = t;
  sl = __fadd_rn(sl, __fadd_rn(err, pe));
}

}  // namespace pdfgb
