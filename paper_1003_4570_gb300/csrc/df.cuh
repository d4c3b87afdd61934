// Double-float arithmetic: a value is an FP32 pair (hi, lo) with value = hi + lo (about 48
// significant bits).  A product a*b is formed exactly in its leading part (p = fl(a.hi b.hi),
// e = fma(a.hi, b.hi, -p); Dekker 1971) plus the cross terms; it is added to a running (S, C)
// pair with Knuth's TwoSum, the rounding error of the sum going into C.  The _rn intrinsics keep
// the compiler from contracting the additions into FMAs, which would break the error-free
// transformations.
#pragma once
#include <cuda_runtime.h>

__device__ __forceinline__ void df_mac(float& S, float& C, float2 a, float2 b) {
  const float p = __fmul_rn(a.x, b.x);
  float e = __fmaf_rn(a.x, b.x, -p);
  e = __fmaf_rn(a.x, b.y, e);
  e = __fmaf_rn(a.y, b.x, e);
  const float s = __fadd_rn(S, p);
  const float bb = __fsub_rn(s, S);
  const float t = __fadd_rn(__fsub_rn(S, __fsub_rn(s, bb)), __fsub_rn(p, bb));
  C = __fadd_rn(C, __fadd_rn(t, e));
  S = s;
}
__device__ __forceinline__ float2 df_norm(float S, float C) {
  const float h = __fadd_rn(S, C);
  return make_float2(h, __fsub_rn(C, __fsub_rn(h, S)));
}
__device__ __forceinline__ float2 df_add(float2 a, float2 b) {
  const float s = __fadd_rn(a.x, b.x);
  const float bb = __fsub_rn(s, a.x);
  const float t = __fadd_rn(__fsub_rn(a.x, __fsub_rn(s, bb)), __fsub_rn(b.x, bb));
  return df_norm(s, __fadd_rn(t, __fadd_rn(a.y, b.y)));
}
__device__ __forceinline__ float2 df_from_double(double v) {
  const float hi = __double2float_rn(v);
  return make_float2(hi, __double2float_rn(v - (double)hi));
}
__device__ __forceinline__ double df_to_double(float2 v) { return (double)v.x + (double)v.y; }
