// Double-float ("dd") arithmetic on pairs of FP32 values (hi + lo, |lo| <=
// ulp(hi)/2), about 48 significant bits.  On this GPU the FP32 pipes are ~70x
// faster than FP64, so the split path's per-element work (recombination of
// slice products, denominators, contravariant combinations, slicing) runs in
// dd arithmetic built from error-free transformations: two-sum (Knuth) and
// two-product via fused multiply-add (Dekker/Ogita-Rump-Oishi).
#pragma once
#include <cuda_runtime.h>

namespace cc3 {
namespace dd {

struct df {
  float hi, lo;
};

__device__ __forceinline__ df two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}
__device__ __forceinline__ df fast_two_sum(float a, float b) {  // |a| >= |b|
  float s = __fadd_rn(a, b);
  float e = __fsub_rn(b, __fsub_rn(s, a));
  return {s, e};
}
__device__ __forceinline__ df add(df a, df b) {
  df s = two_sum(a.hi, b.hi);
  df t = two_sum(a.lo, b.lo);
  s.lo = __fadd_rn(s.lo, t.hi);
  s = fast_two_sum(s.hi, s.lo);
  s.lo = __fadd_rn(s.lo, t.lo);
  return fast_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ df add_f(df a, float b) {
  df s = two_sum(a.hi, b);
  s.lo = __fadd_rn(s.lo, a.lo);
  return fast_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ df mul_f(df a, float b) {
  float p = __fmul_rn(a.hi, b);
  float e = __fmaf_rn(a.hi, b, -p);
  e = __fmaf_rn(a.lo, b, e);
  return fast_two_sum(p, e);
}
__device__ __forceinline__ df mul(df a, df b) {
  float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return fast_two_sum(p, e);
}
// a / b by long division on the quotient: three partial quotients, each
// from the remainder of the previous ones (formed in dd arithmetic) times an
// approximate reciprocal of b.hi.  Each step shrinks the remainder by the
// reciprocal's relative error (~2^-22 for the hardware approximation), so
// the quotient is accurate to the dd arithmetic (~2^-46 relative); the
// reciprocal's last bits do not matter.  |b.hi| must be a normal number.
__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ df div(df a, df b) {
  const float rb = rcp_approx(b.hi);
  const float q1 = a.hi * rb;
  df p = mul_f(b, q1);
  df r = add(a, df{-p.hi, -p.lo});
  const float q2 = r.hi * rb;
  p = mul_f(b, q2);
  r = add(r, df{-p.hi, -p.lo});
  const float q3 = r.hi * rb;
  const df q = fast_two_sum(q1, q2);
  return add_f(q, q3);
}
__device__ __forceinline__ df scale(df a, float s) {  // s a power of two
  return {a.hi * s, a.lo * s};
}
__device__ __forceinline__ df neg(df a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ double to_double(df a) {
  return (double)a.hi + (double)a.lo;
}
__host__ __device__ inline df from_double_host(double x) {
  float h = (float)x;
  float l = (float)(x - (double)h);
  return {h, l};
}

}  // namespace dd
}  // namespace cc3
