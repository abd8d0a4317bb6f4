// irs_df.cuh -- double-float ("double-word") arithmetic on the FP32 pipes for
// the far-field convolution (FFTs and M2L).  A value is the unevaluated sum
// hi + lo of two floats with |lo| <= ulp(hi)/2: 48 significant bits.  GB300
// runs FP64 at 1/64 of its FP32 rate, and a double-float multiply-add costs
// ~30 FP32 operations, so the convolution moves to the FP32 pipes.
//
// The building blocks are the error-free transformations of Knuth (TwoSum),
// Dekker (Fast2Sum) and the FMA form of TwoProd; the sums and products follow
// the "sloppy" double-word addition and the double-word x double-word
// product of Joldes, Muller and Popescu (ACM TOMS 44, 2017), whose relative
// error is a few 2^-48 in the normwise sense an FFT needs.  Every operation
// goes through __fadd_rn / __fmul_rn / __fmaf_rn, so that the compiler cannot
// contract or reorder the exact-rounding steps.
#pragma once

#include <cuda_runtime.h>

namespace irs {

__device__ __forceinline__ void df_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// |a| >= |b| (or a == 0)
__device__ __forceinline__ void df_fast_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}

// x + y (sloppy double-word addition)
__device__ __forceinline__ float2 df_add(float2 x, float2 y) {
  float s, e, h, l;
  df_two_sum(x.x, y.x, s, e);
  e = __fadd_rn(e, __fadd_rn(x.y, y.y));
  df_fast_two_sum(s, e, h, l);
  return make_float2(h, l);
}

__device__ __forceinline__ float2 df_neg(float2 x) { return make_float2(-x.x, -x.y); }

__device__ __forceinline__ float2 df_sub(float2 x, float2 y) { return df_add(x, df_neg(y)); }

// x * y
__device__ __forceinline__ float2 df_mul(float2 x, float2 y) {
  const float p = __fmul_rn(x.x, y.x);
  float e = __fmaf_rn(x.x, y.x, -p);
  e = __fmaf_rn(x.x, y.y, e);
  e = __fmaf_rn(x.y, y.x, e);
  float h, l;
  df_fast_two_sum(p, e, h, l);
  return make_float2(h, l);
}

// a*b + s*c*d for s = +-1: one rounding pass for a complex product's part
__device__ __forceinline__ float2 df_dot2(float2 a, float2 b, float2 c, float2 d, float sgn) {
  const float p1 = __fmul_rn(a.x, b.x);
  float e1 = __fmaf_rn(a.x, b.x, -p1);
  e1 = __fmaf_rn(a.x, b.y, e1);
  e1 = __fmaf_rn(a.y, b.x, e1);
  const float ch = sgn * c.x, cl = sgn * c.y;  // exact sign flips
  const float p2 = __fmul_rn(ch, d.x);
  float e2 = __fmaf_rn(ch, d.x, -p2);
  e2 = __fmaf_rn(ch, d.y, e2);
  e2 = __fmaf_rn(cl, d.x, e2);
  float s, t, h, l;
  df_two_sum(p1, p2, s, t);
  t = __fadd_rn(t, __fadd_rn(e1, e2));
  df_fast_two_sum(s, t, h, l);
  return make_float2(h, l);
}

// Complex double-float, stored as float4 (re.hi, re.lo, im.hi, im.lo).
__device__ __forceinline__ float2 dfc_re(float4 z) { return make_float2(z.x, z.y); }
__device__ __forceinline__ float2 dfc_im(float4 z) { return make_float2(z.z, z.w); }
__device__ __forceinline__ float4 dfc_make(float2 re, float2 im) { return make_float4(re.x, re.y, im.x, im.y); }

__device__ __forceinline__ float4 dfc_mul(float4 a, float4 b) {
  const float2 ar = dfc_re(a), ai = dfc_im(a), br = dfc_re(b), bi = dfc_im(b);
  return dfc_make(df_dot2(ar, br, ai, bi, -1.0f), df_dot2(ar, bi, ai, br, 1.0f));
}

__device__ __forceinline__ float4 dfc_add(float4 a, float4 b) {
  return dfc_make(df_add(dfc_re(a), dfc_re(b)), df_add(dfc_im(a), dfc_im(b)));
}

__device__ __forceinline__ float4 dfc_sub(float4 a, float4 b) {
  return dfc_make(df_sub(dfc_re(a), dfc_re(b)), df_sub(dfc_im(a), dfc_im(b)));
}

// x * s for a double-float real s
__device__ __forceinline__ float4 dfc_scale(float4 a, float2 s) {
  return dfc_make(df_mul(dfc_re(a), s), df_mul(dfc_im(a), s));
}

// FP64 <-> double-float
__host__ __device__ __forceinline__ float2 df_from_double(double x) {
  const float h = (float)x;
  return make_float2(h, (float)(x - (double)h));
}
__host__ __device__ __forceinline__ double df_to_double(float2 x) { return (double)x.x + (double)x.y; }
__host__ __device__ __forceinline__ float4 dfc_from_double(double re, double im) {
  const float2 r = df_from_double(re), i = df_from_double(im);
  return make_float4(r.x, r.y, i.x, i.y);
}

}  // namespace irs
