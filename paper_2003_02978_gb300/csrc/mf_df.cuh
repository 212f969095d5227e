// Double-float ("float-float") arithmetic on the FP32 pipes.
//
// A value is the unevaluated sum hi + lo of two floats (|lo| <= ulp(hi)/2),
// about 48 significant bits.  Built from the error-free transformations of
// Knuth (TwoSum), Dekker (Fast2Sum) and the FMA form of Dekker's TwoProduct;
// reciprocal and square root refine the float32 estimate with one Newton
// step evaluated in double-float.  On GB300 the FP64 pipe runs at 1/64 of
// the FP32 rate with a long dependent latency, so the small dense linear
// algebra of the background model (assembly, Cholesky, triangular
// inversion, solves) runs in this arithmetic instead.
//
// Must not be compiled with fast-math: the transformations rely on IEEE
// round-to-nearest float additions in program order.
#pragma once
#include <cuda_runtime.h>

namespace mf {

struct df {
  float hi, lo;
};

__device__ __forceinline__ df df_make(float h, float l = 0.f) { return df{h, l}; }

// s + e == a + b exactly (Knuth)
__device__ __forceinline__ df two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return df{s, e};
}
// requires |a| >= |b| (Dekker)
__device__ __forceinline__ df fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float e = __fsub_rn(b, __fsub_rn(s, a));
  return df{s, e};
}
// p + e == a * b exactly (FMA form of Dekker's product)
__device__ __forceinline__ df two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  const float e = fmaf(a, b, -p);
  return df{p, e};
}

__device__ __forceinline__ df df_add(df x, df y) {
  df s = two_sum(x.hi, y.hi);
  const df t = two_sum(x.lo, y.lo);
  s.lo = __fadd_rn(s.lo, t.hi);
  s = fast_two_sum(s.hi, s.lo);
  s.lo = __fadd_rn(s.lo, t.lo);
  return fast_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ df df_neg(df x) { return df{-x.hi, -x.lo}; }
__device__ __forceinline__ df df_sub(df x, df y) { return df_add(x, df_neg(y)); }

// add a float to a double-float
__device__ __forceinline__ df df_addf(df x, float y) {
  df s = two_sum(x.hi, y);
  s.lo = __fadd_rn(s.lo, x.lo);
  return fast_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ df df_mul(df x, df y) {
  df p = two_prod(x.hi, y.hi);
  p.lo = fmaf(x.hi, y.lo, p.lo);
  p.lo = fmaf(x.lo, y.hi, p.lo);
  return fast_two_sum(p.hi, p.lo);
}
__device__ __forceinline__ df df_mulf(df x, float y) {
  df p = two_prod(x.hi, y);
  p.lo = fmaf(x.lo, y, p.lo);
  return fast_two_sum(p.hi, p.lo);
}
// a * b + c
__device__ __forceinline__ df df_fma(df a, df b, df c) { return df_add(df_mul(a, b), c); }

// 1/x: float32 estimate r, then r + r (1 - x r) in double-float (Newton)
__device__ __forceinline__ df df_recip(df x) {
  const float r = 1.0f / x.hi;
  const df e = df_sub(df{1.f, 0.f}, df_mulf(x, r));
  return df_add(df{r, 0.f}, df_mulf(e, r));
}
__device__ __forceinline__ df df_div(df a, df b) { return df_mul(a, df_recip(b)); }

// 1/sqrt(x), x > 0: float32 estimate r, then r + r (1 - x r^2) / 2 (Newton)
__device__ __forceinline__ df df_rsqrt(df x) {
  const float r = rsqrtf(x.hi);
  const df xr2 = df_mulf(df_mulf(x, r), r);
  const df e = df_sub(df{1.f, 0.f}, xr2);
  return df_add(df{r, 0.f}, df_mulf(e, 0.5f * r));
}

__device__ __forceinline__ df df_from_double(double d) {
  const float h = __double2float_rn(d);
  const float l = __double2float_rn(d - (double)h);
  return df{h, l};
}
__device__ __forceinline__ double df_to_double(df x) { return (double)x.hi + (double)x.lo; }
__device__ __forceinline__ float df_to_float(df x) { return __fadd_rn(x.hi, x.lo); }

__device__ __forceinline__ bool df_isfinite(df x) { return isfinite(x.hi) && isfinite(x.lo); }

}  // namespace mf
