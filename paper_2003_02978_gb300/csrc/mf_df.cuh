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

// A double-float matrix in shared memory stored as two float planes (hi at
// h[i * ld + j], lo one plane further), so that adjacent elements of a row
// load as float2 pairs for the packed arithmetic below.  ld is even (a
// multiple of 4, with a 16-byte aligned base, for the float4 loads).
struct DfMat {
  float* h;
  int ld;
  int plane;  // float offset of the lo plane
  __device__ __forceinline__ df get(int i, int j) const {
    return df{h[i * ld + j], h[plane + i * ld + j]};
  }
  __device__ __forceinline__ void set(int i, int j, df v) const {
    h[i * ld + j] = v.hi;
    h[plane + i * ld + j] = v.lo;
  }
  // elements (i, j) and (i, j + 1), j even
  __device__ __forceinline__ float2 hi2(int i, int j) const {
    return *reinterpret_cast<const float2*>(h + i * ld + j);
  }
  __device__ __forceinline__ float2 lo2(int i, int j) const {
    return *reinterpret_cast<const float2*>(h + plane + i * ld + j);
  }
  __device__ __forceinline__ void set2(int i, int j, float2 hi, float2 lo) const {
    *reinterpret_cast<float2*>(h + i * ld + j) = hi;
    *reinterpret_cast<float2*>(h + plane + i * ld + j) = lo;
  }
  // elements (i, j .. j + 3), j and ld multiples of 4, plane a multiple of 4
  __device__ __forceinline__ float4 hi4(int i, int j) const {
    return *reinterpret_cast<const float4*>(h + i * ld + j);
  }
  __device__ __forceinline__ float4 lo4(int i, int j) const {
    return *reinterpret_cast<const float4*>(h + plane + i * ld + j);
  }
};

// Packed pairs of double-floats (hi and lo as float2), on the fma.rn.f32x2 /
// add.rn.f32x2 / mul.rn.f32x2 instructions: the same error-free
// transformations per element as above.
__device__ __forceinline__ float2 f2(float v) { return make_float2(v, v); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
  return __ffma2_rn(b, make_float2(-1.f, -1.f), a);  // a - b, exact negation
}
// c - w * a for a packed pair a (hi ah, lo al) and one double-float w given
// as (w.hi, -w.hi, w.lo): the product's error terms are formed exactly, its
// sum with c by TwoSum of the high parts and a plain float sum of the low
// parts (error <= about 2^-47 (|c| + |w a|), the bound the factorisations'
// backward error analysis uses).
__device__ __forceinline__ void df2_fnma(float2& ch, float2& cl, float wh, float wnh, float wl,
                                         float2 ah, float2 al) {
  const float2 pn = __fmul2_rn(f2(wnh), ah);            // -p, p = fl(w.hi * a.hi)
  float2 pe = __ffma2_rn(f2(wh), ah, pn);               // w.hi * a.hi - p (exact)
  pe = __ffma2_rn(f2(wh), al, pe);
  pe = __ffma2_rn(f2(wl), ah, pe);                      // w a = p + pe
  const float2 s = __fadd2_rn(ch, pn);                  // TwoSum(c.hi, -p)
  const float2 bb = sub2(s, ch);
  const float2 e = __fadd2_rn(sub2(ch, sub2(s, bb)), sub2(pn, bb));
  const float2 lo = __fadd2_rn(e, sub2(cl, pe));
  ch = __fadd2_rn(s, lo);                               // Fast2Sum
  cl = sub2(lo, sub2(ch, s));
}
// packed double-float product by one double-float w: (ah, al) * w
__device__ __forceinline__ void df2_mul1(float2& ah, float2& al, df w) {
  const float2 p = __fmul2_rn(ah, f2(w.hi));
  float2 e = __ffma2_rn(ah, f2(w.hi), __fmul2_rn(p, f2(-1.f)));
  e = __ffma2_rn(ah, f2(w.lo), e);
  e = __ffma2_rn(al, f2(w.hi), e);
  ah = __fadd2_rn(p, e);
  al = sub2(e, sub2(ah, p));
}

}  // namespace mf
