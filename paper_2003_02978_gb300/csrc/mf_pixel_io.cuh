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

}  // namespace mf
