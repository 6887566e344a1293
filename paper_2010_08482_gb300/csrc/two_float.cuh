// Two-float arithmetic on the FP32 pipe (CTQ_F32X2), shared by the
// shared-memory and the large-block float64 kernels.
#pragma once

#include <cuda_runtime.h>

namespace ctq {
namespace tf2 {

// Two-float numbers (CTQ_F32X2): x = hi + lo with two float32 words, about
// 48 significant bits, multiplied and added on the FP32 pipe with the
// error-free transformations of Dekker (the product's rounding error as
// fmaf(a, b, -a b)) and Knuth (TwoSum).  The complex form keeps (re, im).
struct DF {
  float hi, lo;
};
struct __align__(16) CDF {
  DF re, im;
};

// ---- two-float arithmetic (no contraction: every step is an explicit
// round-to-nearest intrinsic)
__device__ __forceinline__ DF df_split(double x) {
  const float h = __double2float_rn(x);
  return DF{h, __double2float_rn(x - double(h))};
}
__device__ __forceinline__ double df_val(DF a) { return double(a.hi) + double(a.lo); }
__device__ __forceinline__ double2 df_val(CDF a) { return make_double2(df_val(a.re), df_val(a.im)); }
// acc += f y: the product's and the sum's rounding errors are gathered in
// acc.lo, which df_finish folds back (renormalisation) once per output.
__device__ __forceinline__ void df_fma(DF& acc, float fh, float fl, DF y) {
  const float p = __fmul_rn(fh, y.hi);
  float e = __fmaf_rn(fh, y.hi, -p);
  e = __fmaf_rn(fh, y.lo, e);
  e = __fmaf_rn(fl, y.hi, e);
  const float s = __fadd_rn(acc.hi, p);
  const float bp = __fsub_rn(s, acc.hi);
  const float err = __fadd_rn(__fsub_rn(acc.hi, __fsub_rn(s, bp)), __fsub_rn(p, bp));
  acc.hi = s;
  acc.lo = __fadd_rn(acc.lo, __fadd_rn(err, e));
}
constexpr int X2_RENORM = 4;  // two-float terms between renormalisations
__device__ __forceinline__ void fma_acc(DF& acc, DF f, DF y) { df_fma(acc, f.hi, f.lo, y); }
__device__ __forceinline__ void fma_acc(CDF& acc, CDF f, CDF y) {
  df_fma(acc.re, f.re.hi, f.re.lo, y.re);
  df_fma(acc.re, -f.im.hi, -f.im.lo, y.im);
  df_fma(acc.im, f.re.hi, f.re.lo, y.im);
  df_fma(acc.im, f.im.hi, f.im.lo, y.re);
}
__device__ __forceinline__ void df_norm(DF& a) {
  const float s = __fadd_rn(a.hi, a.lo);
  a.lo = __fsub_rn(a.lo, __fsub_rn(s, a.hi));
  a.hi = s;
}
__device__ __forceinline__ void finish(DF& a) { df_norm(a); }
// a += b for normalised two-float numbers (TwoSum of the high words, low
// words added to its error, renormalised)
__device__ __forceinline__ void add_into(DF& a, DF b) {
  const float s = __fadd_rn(a.hi, b.hi);
  const float bp = __fsub_rn(s, a.hi);
  const float err = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bp)), __fsub_rn(b.hi, bp));
  a.hi = s;
  a.lo = __fadd_rn(err, __fadd_rn(a.lo, b.lo));
  df_norm(a);
}
__device__ __forceinline__ void add_into(CDF& a, CDF b) {
  add_into(a.re, b.re);
  add_into(a.im, b.im);
}
__device__ __forceinline__ void finish(CDF& a) {
  df_norm(a.re);
  df_norm(a.im);
}
__device__ __forceinline__ DF df_mul(DF a, DF b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  const float s = __fadd_rn(p, e);
  return DF{s, __fsub_rn(e, __fsub_rn(s, p))};
}
__device__ __forceinline__ DF operator*(DF a, DF b) { return df_mul(a, b); }
__device__ __forceinline__ CDF operator*(DF a, CDF b) { return CDF{df_mul(a, b.re), df_mul(a, b.im)}; }
__device__ __forceinline__ DF operator*(double a, DF b) { return df_mul(df_split(a), b); }
__device__ __forceinline__ CDF operator*(double a, CDF b) { return df_split(a) * b; }
__device__ __forceinline__ void zero(DF& v) { v = DF{0.f, 0.f}; }
__device__ __forceinline__ void zero(CDF& v) { v = CDF{DF{0.f, 0.f}, DF{0.f, 0.f}}; }
// exponent key on the float64 scale (bias 1023), so that the rescale logic
// is shared: 0 for a zero or subnormal high word
__device__ __forceinline__ int exp_key(DF v) {
  const int f = (__float_as_int(v.hi) >> 23) & 0xff;
  return f ? f + (1023 - 127) : 0;
}
__device__ __forceinline__ int exp_key(CDF v) { return max(exp_key(v.re), exp_key(v.im)); }
__device__ __forceinline__ double sq(DF v) { return double(__fmul_rn(v.hi, v.hi)); }
__device__ __forceinline__ double sq(CDF v) { return double(__fmaf_rn(v.re.hi, v.re.hi, __fmul_rn(v.im.hi, v.im.hi))); }

}  // namespace tf2
}  // namespace ctq
