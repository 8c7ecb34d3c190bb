// ff.cuh -- float-float ("double-word") arithmetic on the FP32 pipe.
//
// A value is the unevaluated sum hi + lo of two floats with |lo| <= ulp(hi)/2,
// about 48 significant bits.  GB300 issues FP32 operations at 64 times the
// FP64 rate, so a float-float operation (5 to 20 FP32 instructions) costs a
// fraction of an FP64 one.  The building blocks are the error-free
// transformations of the literature, written here from their definitions:
//   two_sum       Knuth (TAOCP vol. 2, 4.2.2) / Moller (1965): s + e = a + b exactly
//   fast_two_sum  Dekker (1971): the same when |a| >= |b|
//   two_prod      with a fused multiply-add: p + e = a b exactly
// and the double-word algorithms analysed by Joldes, Muller and Popescu
// (ACM TOMS 2017): the "sloppy" sum (relative error bounded when both
// operands have the same sign; absolute error about 2^-47 (|a| + |b|)
// otherwise), the product with the cross terms folded into the FMA, and one
// Newton step in float-float for the reciprocal, the inverse square root
// (seeded by the hardware approximations on the high word) and the square
// root (seeded by the FP32 square root).
//
// Every primitive uses the _rn intrinsics, which the compiler never fuses
// into FMAs, so the error-free transformations stay exact.
#pragma once

#include <cuda_runtime.h>

namespace grmhd {

struct ff {
  float hi, lo;
};

__device__ __forceinline__ float two_sum(float a, float b, float &e) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return s;
}

__device__ __forceinline__ float fast_two_sum(float a, float b, float &e) {
  const float s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
  return s;
}

__device__ __forceinline__ ff ff_make(float hi, float lo) {
  ff r;
  r.hi = fast_two_sum(hi, lo, r.lo);
  return r;
}

// double -> float-float: the high word is x rounded to float, the low word
// the rounded remainder (48 of the 53 bits are kept)
__device__ __forceinline__ ff ff_from(double x) {
  ff r;
  r.hi = __double2float_rn(x);
  r.lo = __double2float_rn(__dsub_rn(x, (double)r.hi));
  return r;
}

__device__ __forceinline__ ff ff_f(float x) {
  ff r;
  r.hi = x;
  r.lo = 0.0f;
  return r;
}

__device__ __forceinline__ double ff_to(ff a) { return __dadd_rn((double)a.hi, (double)a.lo); }

__device__ __forceinline__ ff ff_neg(ff a) {
  ff r;
  r.hi = -a.hi;
  r.lo = -a.lo;
  return r;
}

// exact scaling by a power of two
__device__ __forceinline__ ff ff_ldexp(ff a, float p2) {
  ff r;
  r.hi = __fmul_rn(a.hi, p2);
  r.lo = __fmul_rn(a.lo, p2);
  return r;
}

__device__ __forceinline__ ff ff_add(ff a, ff b) {
  float e;
  const float s = two_sum(a.hi, b.hi, e);
  e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  return ff_make(s, e);
}

__device__ __forceinline__ ff ff_sub(ff a, ff b) { return ff_add(a, ff_neg(b)); }

__device__ __forceinline__ ff ff_add_f(ff a, float b) {
  float e;
  const float s = two_sum(a.hi, b, e);
  e = __fadd_rn(e, a.lo);
  return ff_make(s, e);
}

__device__ __forceinline__ ff ff_mul(ff a, ff b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return ff_make(p, e);
}

__device__ __forceinline__ ff ff_mul_f(ff a, float b) {
  const float p = __fmul_rn(a.hi, b);
  float e = __fmaf_rn(a.hi, b, -p);
  e = __fmaf_rn(a.lo, b, e);
  return ff_make(p, e);
}

__device__ __forceinline__ ff ff_sqr(ff a) {
  const float p = __fmul_rn(a.hi, a.hi);
  float e = __fmaf_rn(a.hi, a.hi, -p);
  e = __fmaf_rn(__fmul_rn(2.0f, a.hi), a.lo, e);
  return ff_make(p, e);
}

// a b + c
__device__ __forceinline__ ff ff_fma(ff a, ff b, ff c) { return ff_add(ff_mul(a, b), c); }

// 1/a: FP32 seed r0 (the hardware approximation, within about an ulp of
// 1/hi; a is never near the float underflow in these bodies, which work in
// scaled units), then r0 + r0 (1 - a r0) with the residual in float-float,
// which squares the seed's relative error
__device__ __forceinline__ ff ff_rcp(ff a) {
  float r0;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r0) : "f"(a.hi));
  const ff res = ff_add_f(ff_neg(ff_mul_f(a, r0)), 1.0f);  // 1 - a r0, small
  return ff_add_f(ff_mul_f(res, r0), r0);
}

__device__ __forceinline__ ff ff_div(ff a, ff b) { return ff_mul(a, ff_rcp(b)); }

// sqrt(a), a >= 0: s0 = sqrtf(hi), then s0 + (a - s0^2) / (2 s0)
__device__ __forceinline__ ff ff_sqrt(ff a) {
  if (!(a.hi > 0.0f)) return ff_f(0.0f);
  const float s0 = __fsqrt_rn(a.hi);
  float e;
  const float p = __fmul_rn(s0, s0);
  e = __fmaf_rn(s0, s0, -p);  // s0^2 = p + e exactly
  const ff d = ff_sub(a, ff_make(p, e));
  return ff_add_f(ff_mul_f(d, __fdiv_rn(0.5f, s0)), s0);
}

// 1/sqrt(a), a > 0: y0 from the hardware approximation of 1/sqrt(hi), then
// y0 + y0 (1 - a y0^2) / 2
__device__ __forceinline__ ff ff_rsqrt(ff a) {
  float y0;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y0) : "f"(a.hi));
  const ff ay = ff_mul_f(ff_mul_f(a, y0), y0);
  const ff res = ff_add_f(ff_neg(ay), 1.0f);
  return ff_add_f(ff_mul_f(res, __fmul_rn(0.5f, y0)), y0);
}

__device__ __forceinline__ bool ff_gt(ff a, ff b) {
  return a.hi > b.hi || (a.hi == b.hi && a.lo > b.lo);
}
__device__ __forceinline__ ff ff_max(ff a, ff b) { return ff_gt(a, b) ? a : b; }
__device__ __forceinline__ ff ff_min(ff a, ff b) { return ff_gt(a, b) ? b : a; }
__device__ __forceinline__ ff ff_abs(ff a) { return (a.hi < 0.0f) ? ff_neg(a) : a; }

}  // namespace grmhd
