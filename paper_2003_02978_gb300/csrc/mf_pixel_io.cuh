// Per-pixel helpers shared by the statistics and pixel kernels, so that both
// compute the split x = rho * ref + e identically.
//
// Two lanes own one pixel: lane e (0 or 1) holds the float4 groups
// f = e + 2 j (j < NJ) of the pixel's band window.  With a pixel row stride
// of B floats (B % 4 == 0) the 8 lanes of a shared-memory phase touch
// distinct bank groups, and the per-pixel dot products need one shuffle.
#pragma once
#include "mf_common.cuh"

namespace mf {

// load the lane's float4 groups of one pixel from shared memory; returns the
// pair's finiteness (both lanes agree)
template <int NJ>
__device__ __forceinline__ bool lds_pixel(const float* px, bool inb, int e, int B4,
                                          float4 (&x)[NJ]) {
  const float4* p4 = reinterpret_cast<const float4*>(px);
  bool fin = true;
#pragma unroll
  for (int j = 0; j < NJ; ++j) {
    const int f = e + 2 * j;
    if (inb && f < B4) {
      x[j] = p4[f];
      fin = fin && finite4(x[j]);
    } else {
      x[j] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
  }
  const int both = __shfl_xor_sync(0xffffffffu, (int)fin, 1) & (int)fin;
  return both != 0;
}

template <int NJ>
__device__ __forceinline__ void sts_pixel(float* px, int e, int B4, const float4 (&x)[NJ]) {
  float4* p4 = reinterpret_cast<float4*>(px);
#pragma unroll
  for (int j = 0; j < NJ; ++j) {
    const int f = e + 2 * j;
    if (f < B4) p4[f] = x[j];
  }
}

// dot over the pair's bands: two partial sums per lane (even / odd groups)
template <int NJ>
__device__ __forceinline__ float pair_dot(const float4 (&x)[NJ], const float4* ref, int e, int B4) {
  float d0 = 0.f, d1 = 0.f;
#pragma unroll
  for (int j = 0; j < NJ; ++j) {
    const int f = e + 2 * j;
    if (f < B4) {
      const float4 m = ref[f];
      float d = (j & 1) ? d1 : d0;
      d = fmaf(x[j].x, m.x, d);
      d = fmaf(x[j].y, m.y, d);
      d = fmaf(x[j].z, m.z, d);
      d = fmaf(x[j].w, m.w, d);
      if (j & 1)
        d1 = d;
      else
        d0 = d;
    }
  }
  const float d = d0 + d1;
  return d + __shfl_xor_sync(0xffffffffu, d, 1);
}

// x <- x - rho * ref  (the residual e_i of the albedo-direction split)
template <int NJ>
__device__ __forceinline__ void split_residual(float4 (&x)[NJ], const float4* ref, float rho,
                                               int e, int B4) {
#pragma unroll
  for (int j = 0; j < NJ; ++j) {
    const int f = e + 2 * j;
    if (f < B4) {
      const float4 m = ref[f];
      x[j].x = fmaf(-rho, m.x, x[j].x);
      x[j].y = fmaf(-rho, m.y, x[j].y);
      x[j].z = fmaf(-rho, m.z, x[j].z);
      x[j].w = fmaf(-rho, m.w, x[j].w);
    }
  }
}

// Packed two-lane float32 arithmetic (fma.rn.f32x2): each instruction does
// the .xy or .zw half of a float4 group, correctly rounded per element.
__device__ __forceinline__ float2 lo2(const float4& v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 hi2(const float4& v) { return make_float2(v.z, v.w); }

// dot over the pair's bands (two packed partial sums per lane, then the
// pair's shuffle).  Any non-finite element of x makes the result non-finite
// (x * 0 is NaN for x = +-Inf or NaN), so the caller's finiteness test of
// the dot replaces a per-element test, for every finite ref.
template <int NJ>
__device__ __forceinline__ float pair_dot2(const float4 (&x)[NJ], const float4 (&ref)[NJ]) {
  float2 d0 = make_float2(0.f, 0.f), d1 = make_float2(0.f, 0.f);
#pragma unroll
  for (int j = 0; j < NJ; ++j) {
    d0 = __ffma2_rn(lo2(x[j]), lo2(ref[j]), d0);
    d1 = __ffma2_rn(hi2(x[j]), hi2(ref[j]), d1);
  }
  const float d = (d0.x + d0.y) + (d1.x + d1.y);
  return d + __shfl_xor_sync(0xffffffffu, d, 1);
}
// x <- x - rho * ref
template <int NJ>
__device__ __forceinline__ void split_residual2(float4 (&x)[NJ], const float4 (&ref)[NJ],
                                                float rho) {
  const float2 m = make_float2(-rho, -rho);
#pragma unroll
  for (int j = 0; j < NJ; ++j) {
    const float2 a = __ffma2_rn(m, lo2(ref[j]), lo2(x[j]));
    const float2 b = __ffma2_rn(m, hi2(ref[j]), hi2(x[j]));
    x[j] = make_float4(a.x, a.y, b.x, b.y);
  }
}
// pair_dot2 / split_residual2 with the reference in shared memory at the
// lane's band groups f = e + 2 j (those past B4 are skipped)
template <int NJ>
__device__ __forceinline__ float pair_dot2s(const float4 (&x)[NJ], const float4* ref, int e, int B4) {
  float2 d0 = make_float2(0.f, 0.f), d1 = make_float2(0.f, 0.f);
#pragma unroll
  for (int j = 0; j < NJ; ++j) {
    const int f = e + 2 * j;
    if (f < B4) {
      const float4 r = ref[f];
      d0 = __ffma2_rn(lo2(x[j]), lo2(r), d0);
      d1 = __ffma2_rn(hi2(x[j]), hi2(r), d1);
    }
  }
  const float d = (d0.x + d0.y) + (d1.x + d1.y);
  return d + __shfl_xor_sync(0xffffffffu, d, 1);
}
template <int NJ>
__device__ __forceinline__ void split_residual2s(float4 (&x)[NJ], const float4* ref, float rho,
                                                 int e, int B4) {
  const float2 m = make_float2(-rho, -rho);
#pragma unroll
  for (int j = 0; j < NJ; ++j) {
    const int f = e + 2 * j;
    if (f < B4) {
      const float4 r = ref[f];
      const float2 a = __ffma2_rn(m, lo2(r), lo2(x[j]));
      const float2 b = __ffma2_rn(m, hi2(r), hi2(x[j]));
      x[j] = make_float4(a.x, a.y, b.x, b.y);
    }
  }
}
// acc <- acc + s * x
template <int NJ>
__device__ __forceinline__ void axpy2(float4 (&acc)[NJ], float s, const float4 (&x)[NJ]) {
  const float2 m = make_float2(s, s);
#pragma unroll
  for (int j = 0; j < NJ; ++j) {
    const float2 a = __ffma2_rn(m, lo2(x[j]), lo2(acc[j]));
    const float2 b = __ffma2_rn(m, hi2(x[j]), hi2(acc[j]));
    acc[j] = make_float4(a.x, a.y, b.x, b.y);
  }
}

}  // namespace mf
