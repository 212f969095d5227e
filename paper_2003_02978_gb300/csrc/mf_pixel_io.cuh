// Per-pixel load and projection helpers shared by the statistics and pixel
// kernels, so that both compute the split x = rho * ref + e identically.
//
// Two lanes own one pixel: lane e (0 or 1) holds the float4 groups
// f = e + 2 j (j < NJ) of the pixel's band window.  A warp therefore covers 16
// pixels per step; every load instruction fetches 16 fully used 32-byte
// sectors, and the per-pixel dot products need one shuffle.
#pragma once
#include "mf_common.cuh"

namespace mf {

template <int NJ>
__device__ __forceinline__ bool load_pixel(const Params& p, int row, int col, bool inb, int e,
                                           float4 (&x)[NJ]) {
  const float4* px = reinterpret_cast<const float4*>(pixel_ptr(p, inb ? row : 0, col));
  bool fin = true;
#pragma unroll
  for (int j = 0; j < NJ; ++j) {
    const int f = e + 2 * j;
    if (inb && f < p.B4) {
      x[j] = __ldg(px + f);
      fin = fin && finite4(x[j]);
    } else {
      x[j] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
  }
  // the pair agrees on finiteness
  const int both = __shfl_xor_sync(0xffffffffu, (int)fin, 1) & (int)fin;
  return both != 0;
}

template <int NJ>
__device__ __forceinline__ float pair_dot(const float4 (&x)[NJ], const float4* ref, int e, int B4) {
  float d = 0.f;
#pragma unroll
  for (int j = 0; j < NJ; ++j) {
    const int f = e + 2 * j;
    if (f < B4) {
      const float4 m = ref[f];
      d = fmaf(x[j].x, m.x, d);
      d = fmaf(x[j].y, m.y, d);
      d = fmaf(x[j].z, m.z, d);
      d = fmaf(x[j].w, m.w, d);
    }
  }
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
