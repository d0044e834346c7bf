// Float-float arithmetic: a value is hi + lo with |lo| <= ulp(hi) / 2, built from
// error-free float32 transforms (two-sum, fma-based product error).  Used where
// float64 would be needed for accuracy but the FP64 pipe (1/64 of FP32 on this
// GPU) would set the pace.
#pragma once

#include <cuda_runtime.h>

namespace {

struct FF {
  float h, l;
};
__device__ __forceinline__ FF ff_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}
__device__ __forceinline__ FF ff_fast(float a, float b) {  // |a| >= |b|
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ FF ff_add(FF a, FF b) {
  const FF s = ff_two_sum(a.h, b.h);
  return ff_fast(s.h, __fadd_rn(s.l, __fadd_rn(a.l, b.l)));
}
__device__ __forceinline__ FF ff_neg(FF a) { return {-a.h, -a.l}; }
__device__ __forceinline__ FF ff_sqr(FF a) {
  const float p = __fmul_rn(a.h, a.h);
  const float e = __fmaf_rn(a.h, a.h, -p);
  return ff_fast(p, __fmaf_rn(__fmul_rn(2.0f, a.h), a.l, e));
}
__device__ __forceinline__ FF ff_mul(FF a, float b) {
  const float p = __fmul_rn(a.h, b);
  const float e = __fmaf_rn(a.h, b, -p);
  return ff_fast(p, __fmaf_rn(a.l, b, e));
}
}  // namespace
