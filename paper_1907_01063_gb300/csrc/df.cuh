// Double-float arithmetic: a value is an unevaluated sum hi + lo of two FP32
// numbers with |lo| <= ulp(hi) / 2, about 48 significant bits.  The error-free
// transformations are Knuth's two-sum, Dekker's fast two-sum (|a| >= |b|) and
// the FMA-based two-product; addition and multiplication follow the usual
// double-double constructions (Hida, Li & Bailey, "Algorithms for quad-double
// precision floating point arithmetic", 2001) with FP32 in place of FP64.
// The round-to-nearest intrinsics keep the compiler from contracting or
// reassociating the transformations.
//
// On GB300 the FP32 pipe is some seventy times faster than the FP64 pipe, so
// elementwise work that needs more than FP32 but less than FP64 accuracy
// (here the squared-exponential covariance of the mixed-precision path) runs
// far faster in double-float.
#pragma once
#include <cuda_runtime.h>

namespace gpc {
namespace dfa {

struct df {
  float hi, lo;
};

__device__ __forceinline__ df two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float v = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, v)), __fsub_rn(b, v));
  return {s, e};
}
__device__ __forceinline__ df fast_two_sum(float a, float b) {  // requires |a| >= |b| or a == 0
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ df two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return {p, __fmaf_rn(a, b, -p)};
}
// accurate sum (cancellation-safe)
__device__ __forceinline__ df add(df a, df b) {
  df s = two_sum(a.hi, b.hi);
  const df t = two_sum(a.lo, b.lo);
  s.lo = __fadd_rn(s.lo, t.hi);
  s = fast_two_sum(s.hi, s.lo);
  s.lo = __fadd_rn(s.lo, t.lo);
  return fast_two_sum(s.hi, s.lo);
}
// sum without the low-part two-sum: accurate when a and b do not cancel
__device__ __forceinline__ df add_same_sign(df a, df b) {
  df s = two_sum(a.hi, b.hi);
  s.lo = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
  return fast_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ df mul(df a, df b) {
  df p = two_prod(a.hi, b.hi);
  p.lo = __fmaf_rn(a.hi, b.lo, p.lo);
  p.lo = __fmaf_rn(a.lo, b.hi, p.lo);
  return fast_two_sum(p.hi, p.lo);
}
__device__ __forceinline__ df neg(df a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ df from_double(double x) {
  const float h = __double2float_rn(x);
  return {h, __double2float_rn(x - (double)h)};
}
__device__ __forceinline__ double to_double(df a) { return (double)a.hi + (double)a.lo; }

// e^{-t} for a double-float t in [0, 80], returned as a double-float mantissa
// m in [sqrt(2)/2, sqrt(2)] and a power of two k (e^{-t} = m 2^k, k in
// [-116, 0]).  Cody & Waite's reduction -t = k ln2 + r with ln2 split into
// three FP32 parts (the first with 15 significant bits, so k * part exactly),
// then e^{r/2} from the Taylor series to degree 10 (|r/2| <= 0.174, remainder
// below 2^-53) evaluated by Horner's rule, squared.  Relative error about 2^-46.
__device__ __forceinline__ df exp_neg(df t, int &k_out) {
  const float kINV_LN2 = 1.44269502162933349609375f;
  const float kLN2_HI = 0x1.62e4p-1f;      // 15 significant bits
  const float kLN2_MID = 0x1.7f7d1cp-20f;
  const float kLN2_LO = 0x1.ef357ap-45f;
  // 1/j! as double-floats, j = 0..10
  const float c_hi[11] = {1.0f, 1.0f, 0.5f, 0x1.555556p-3f, 0x1.555556p-5f, 0x1.111112p-7f,
                          0x1.6c16c2p-10f, 0x1.a01a02p-13f, 0x1.a01a02p-16f, 0x1.71de3ap-19f, 0x1.27e4fcp-22f};
  const float c_lo[11] = {0.0f, 0.0f, 0.0f, -0x1.555556p-28f, -0x1.555556p-30f, -0x1.dddddep-32f,
                          -0x1.27d27ep-35f, -0x1.7f97fap-39f, -0x1.7f97fap-42f, 0x1.55b1ccp-45f, -0x1.10ec14p-47f};
  const df x = neg(t);
  const float k = rintf(__fmul_rn(x.hi, kINV_LN2));
  const float rh = __fsub_rn(x.hi, __fmul_rn(k, kLN2_HI));  // exact: k * kLN2_HI has <= 24 bits
  df r = add(two_sum(rh, x.lo), neg(two_prod(k, kLN2_MID)));
  r = add(r, df{-__fmul_rn(k, kLN2_LO), 0.0f});
  const df s = {__fmul_rn(r.hi, 0.5f), __fmul_rn(r.lo, 0.5f)};
  df p = {c_hi[10], c_lo[10]};
#pragma unroll
  for (int j = 9; j >= 0; --j) p = add(mul(p, s), df{c_hi[j], c_lo[j]});
  p = mul(p, p);
  k_out = (int)k;
  return p;
}

// 2^k as a double for k in [-1022, 1023]
__device__ __forceinline__ double pow2(int k) { return __longlong_as_double((long long)(k + 1023) << 52); }

}  // namespace dfa
}  // namespace gpc
