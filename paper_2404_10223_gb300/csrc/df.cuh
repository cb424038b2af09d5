// Double-float arithmetic: a value is an unevaluated sum hi + lo of two FP32
// numbers (float2 x = hi, y = lo), about 48 significant bits, built from the
// error-free transformations TwoSum (Knuth) and TwoProduct by FMA.  Used where
// GB300's FP32 rate (64x its FP64 rate) makes it cheaper than FP64.  Every
// operation uses explicitly rounded intrinsics so that no multiply-add
// contraction changes an error term.
#pragma once
#include <cuda_runtime.h>

namespace tnqe {
namespace dfa {

__device__ __forceinline__ float2 from_double(double v) {
  const float h = __double2float_rn(v);
  return make_float2(h, __double2float_rn(v - (double)h));
}
__device__ __forceinline__ double to_double(float2 a) { return (double)a.x + (double)a.y; }

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ float2 fast_two_sum(float a, float b) {   // |a| >= |b| or a == 0
  const float s = __fadd_rn(a, b);
  return make_float2(s, __fsub_rn(b, __fsub_rn(s, a)));
}
__device__ __forceinline__ float2 mul(float2 a, float2 b) {
  const float p = __fmul_rn(a.x, b.x);
  float e = fmaf(a.x, b.x, -p);
  e = __fadd_rn(e, __fadd_rn(__fmul_rn(a.x, b.y), __fmul_rn(a.y, b.x)));
  return fast_two_sum(p, e);
}
__device__ __forceinline__ float2 add(float2 a, float2 b) {
  float s, e;
  two_sum(a.x, b.x, s, e);
  e = __fadd_rn(e, __fadd_rn(a.y, b.y));
  return fast_two_sum(s, e);
}
// c + a b
__device__ __forceinline__ float2 fma(float2 a, float2 b, float2 c) { return add(mul(a, b), c); }

}  // namespace dfa
}  // namespace tnqe
