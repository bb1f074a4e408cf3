// Float-float ("double-single") arithmetic: a value is the unevaluated sum h + l of two floats
// with |l| <= ulp(h)/2, about 48 significant bits. The mixed-precision path keeps the state and
// the stage residuals in this form, so the time update needs no FP64 instructions (GB300 issues
// FP64 at 1/64 of the FP32 rate). Error-free transformations after Knuth (TwoSum), Dekker
// (Fast2Sum) and the FMA form of TwoProduct; the explicit _rn intrinsics keep the compiler from
// contracting or reassociating them.
#pragma once

#include <cuda_runtime.h>

namespace gks {

struct __align__(8) ff {
  float h, l;
};

// s + e = a + b exactly (any a, b)
__device__ __forceinline__ ff two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}
// s + e = a + b exactly when |a| >= |b| (or a = 0)
__device__ __forceinline__ ff fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
// x + y with both parts' rounding errors carried (accurate also under cancellation)
__device__ __forceinline__ ff ff_add(ff x, ff y) {
  ff s = two_sum(x.h, y.h);
  const ff t = two_sum(x.l, y.l);
  s = fast_two_sum(s.h, __fadd_rn(s.l, t.h));
  return fast_two_sum(s.h, __fadd_rn(s.l, t.l));
}
__device__ __forceinline__ ff ff_mul(ff x, ff y) {
  const float p = __fmul_rn(x.h, y.h);
  float e = __fmaf_rn(x.h, y.h, -p);  // exact rounding error of p
  e = __fmaf_rn(x.h, y.l, e);
  e = __fmaf_rn(x.l, y.h, e);
  return fast_two_sum(p, e);
}
__device__ __forceinline__ ff ff_twice(ff x) { return {2.f * x.h, 2.f * x.l}; }  // exact
// Nearest float-float of a double (host or device).
__host__ __device__ __forceinline__ ff ff_from(double x) {
  const float h = (float)x;
  return {h, (float)(x - (double)h)};
}
__device__ __forceinline__ double ff_to_double(ff x) { return (double)x.h + (double)x.l; }

}  // namespace gks
