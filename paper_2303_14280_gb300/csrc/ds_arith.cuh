// Double-FP32 ("ds") arithmetic: a value is the unevaluated sum hi + lo of two
// floats with |lo| <= ulp(hi) / 2, about 48 significant bits.  Built from the
// error-free transformations of floating-point arithmetic:
//   TwoSum (Knuth):      s + e = a + b exactly, 6 FP32 operations;
//   FastTwoSum (Dekker): the same when |a| >= |b|, 3 operations;
//   TwoProd:             p + e = a b exactly with one FMA, 2 operations.
// Addition adds the low parts into the TwoSum error and renormalises (11
// operations, error ~2^-46 (|x| + |y|)); multiplication keeps the cross terms
// (7 operations, ~2^-46 relative); a fused multiply-add is the product
// followed by the addition (15 operations).  Every step uses the _rn
// intrinsics so that the compiler neither contracts nor reorders them.
//
// On GB300 the FP32 pipe issues 64x the FP64 rate, so ds arithmetic runs
// several times faster than FP64 at a precision (~1e-14 relative) far below
// what the K tolerance needs.
#pragma once

#include <cuda_runtime.h>

namespace snk {

// the ds overload of fma below must not hide the FP64 / FP32 ones
using ::fma;

struct ds {
  float hi, lo;
};

__device__ __forceinline__ ds ds_make(float hi, float lo) {
  ds r;
  r.hi = hi;
  r.lo = lo;
  return r;
}

__device__ __forceinline__ ds ds_from(double v) {
  const float h = __double2float_rn(v);
  return ds_make(h, __double2float_rn(v - (double)h));
}

__device__ __forceinline__ double ds_to(ds a) { return (double)a.hi + (double)a.lo; }

__device__ __forceinline__ ds ds_fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return ds_make(s, __fsub_rn(b, __fsub_rn(s, a)));
}

__device__ __forceinline__ ds operator+(ds x, ds y) {
  const float s = __fadd_rn(x.hi, y.hi);
  const float bb = __fsub_rn(s, x.hi);
  const float e = __fadd_rn(__fsub_rn(x.hi, __fsub_rn(s, bb)), __fsub_rn(y.hi, bb));
  return ds_fast_two_sum(s, __fadd_rn(e, __fadd_rn(x.lo, y.lo)));
}

__device__ __forceinline__ ds operator-(ds x) { return ds_make(-x.hi, -x.lo); }
__device__ __forceinline__ ds operator-(ds x, ds y) { return x + (-y); }
__device__ __forceinline__ ds& operator+=(ds& x, ds y) {
  x = x + y;
  return x;
}

__device__ __forceinline__ ds operator*(ds x, ds y) {
  const float p = __fmul_rn(x.hi, y.hi);
  float e = __fmaf_rn(x.hi, y.hi, -p);
  e = __fmaf_rn(x.hi, y.lo, e);
  e = __fmaf_rn(x.lo, y.hi, e);
  return ds_fast_two_sum(p, e);
}

// x times an exactly representable float
__device__ __forceinline__ ds operator*(ds x, float s) {
  const float p = __fmul_rn(x.hi, s);
  float e = __fmaf_rn(x.hi, s, -p);
  e = __fmaf_rn(x.lo, s, e);
  return ds_fast_two_sum(p, e);
}

__device__ __forceinline__ ds fma(ds x, ds y, ds z) {
  const float p = __fmul_rn(x.hi, y.hi);
  float e = __fmaf_rn(x.hi, y.hi, -p);
  e = __fmaf_rn(x.hi, y.lo, e);
  e = __fmaf_rn(x.lo, y.hi, e);
  const float s = __fadd_rn(p, z.hi);
  const float bb = __fsub_rn(s, p);
  const float t = __fadd_rn(__fsub_rn(p, __fsub_rn(s, bb)), __fsub_rn(z.hi, bb));
  return ds_fast_two_sum(s, __fadd_rn(t, __fadd_rn(e, z.lo)));
}

// 1 / sqrt(t) for t > 0: the FP32 estimate refined by one Newton step in ds
// (the relative error squares: ~1e-14).
__device__ __forceinline__ ds ds_rsqrt(ds t) {
  const float r0 = rsqrtf(t.hi);
  const ds y = (t * r0) * r0;                       // t r0^2 = 1 - d
  const ds h = ds_make(1.0f, 0.0f) - y;              // d
  return ds_make(r0, 0.0f) + (ds_make(r0, 0.0f) * h) * 0.5f;
}

}  // namespace snk
