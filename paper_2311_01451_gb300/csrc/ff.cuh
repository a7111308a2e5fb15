// Float-float arithmetic on the FP32 pipe: an unevaluated sum h + l of two FP32 numbers with
// |l| <= ulp(h)/2 (48 significant bits).  Error-free transformations: Knuth's TwoSum, Dekker's
// FastTwoSum (|a| >= |b|) and TwoProduct through the fused multiply-add.
#pragma once
#include <cuda_runtime.h>

namespace rsrs {

struct ffv {
  float h, l;
};

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}
__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
  p = __fmul_rn(a, b);
  e = __fmaf_rn(a, b, -p);
}
// a + b with both pairs' rounding errors kept (Bailey's accurate addition).
__device__ __forceinline__ ffv ff_add(ffv a, ffv b) {
  float s, e, t, f;
  two_sum(a.h, b.h, s, e);
  two_sum(a.l, b.l, t, f);
  e = __fadd_rn(e, t);
  fast_two_sum(s, e, s, e);
  e = __fadd_rn(e, f);
  fast_two_sum(s, e, s, e);
  return {s, e};
}

}  // namespace rsrs
