// Statistics kernel: second moments of the background of each partition.
//
// Fig. 1 (Algorithm AlbedoReWeightL1Filter) initialises mu^0 = (1/N) sum L_i
// and C^0 = (1/N) sum (L_i - mu^0)(L_i - mu^0)^T (outer product, as in
// Eq. (11)); the literal schedule recomputes C^k = (1/N) sum d_i d_i^T with
// d_i = L_i - r_i alpha_i^{k-1} t(mu^k) - mu^k at every iteration.
//
// One CTA streams one detector column over a chunk of rows: a TMA box of 128
// rows x B bands per stage, double buffered on mbarriers.  Each pixel is
// split along a reference direction m (the first valid pixel of the
// partition at initialisation, mu^0 afterwards):
//   x_i = rho_i m + e_i,  rho_i = x_i.m / m.m,
// which removes the large albedo component (Sec. II-C) from what is
// accumulated in float32.  The CTA forms the augmented second moments of
//   [e_i, a_i, b_i, 1],  a_i = rho_i - 1,  b_i = -r_i alpha_i^{k-1},
// a symmetric (B+3)x(B+3) product in 4x4 register blocks, folded every 32
// pixels into double-float (TwoSum) accumulators, and writes them out.  The
// solve kernel reduces them and assembles C exactly.
#include "mf_common.cuh"
#include "mf_pixel_io.cuh"
#include "mf_tma.cuh"
#include "../../include/mf.h"

namespace mf {

namespace {
constexpr int kFold = 32;

__device__ __forceinline__ void two_sum_acc(float& hi, float& lo, float x) {
  const float s = __fadd_rn(hi, x);
  const float bp = __fsub_rn(s, hi);
  const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(x, bp));
  hi = s;
  lo = __fadd_rn(lo, err);
}

struct StatSmem {
  size_t stage_bytes, stages_off, coef_off, acc_off, bar_off, total;
};
// stages | coefficients [a, b, 1, 0] | double-float accumulators | barriers
__host__ __device__ inline StatSmem stat_layout(int B) {
  StatSmem L;
  const int nb = (B + 4) / 4;
  const size_t nblk = (size_t)nb * (nb + 1) / 2;
  L.stage_bytes = (size_t)kStatRows * B * sizeof(float);
  L.stages_off = 0;
  L.coef_off = 2 * L.stage_bytes;
  L.acc_off = L.coef_off + 2 * (size_t)kStatRows * 4 * sizeof(float);
  L.bar_off = L.acc_off + nblk * 32 * sizeof(float);
  L.total = L.bar_off + 4 * sizeof(uint64_t);
  return L;
}
}  // namespace

size_t stats_smem_bytes(int B) { return stat_layout(B).total + 128; }

template <int NJ>
__global__ void __launch_bounds__(kThreads) stats_kernel(const __grid_constant__ CUtensorMap map,
                                                         Params p, int mode, int pass) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(16) float s_ref[kMaxB];
  __shared__ float s_inv_ref2;
  __shared__ int s_pilot, s_abort;

  const StatItem it = stat_item(p, blockIdx.x);
  const LineInfo line = p.lines[it.line];
  // literal schedule: lines whose iterations are done take no part
  if (mode == STAT_LITERAL && pass > line.n_iter) return;
  const int c = it.c;
  const int chunk = it.chunk;
  const int part = part_of(p, it.line, c);
  const int c0 = part_col0(p, part);
  const int ncp = part_ncols(p, part);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int B = p.B, B4 = p.B4, BA = p.BA;
  const StatSmem L = stat_layout(B);
  float* stage[2] = {reinterpret_cast<float*>(smem_raw + L.stages_off),
                     reinterpret_cast<float*>(smem_raw + L.stages_off + L.stage_bytes)};
  float4* coef[2] = {reinterpret_cast<float4*>(smem_raw + L.coef_off),
                     reinterpret_cast<float4*>(smem_raw + L.coef_off) + kStatRows};
  uint64_t* full = reinterpret_cast<uint64_t*>(smem_raw + L.bar_off);

  const int r_beg = it.r_beg;
  const int r_end = it.r_end;
  const int nst = (r_end - r_beg + kStatRows - 1) / kStatRows;
  const uint32_t box_bytes = (uint32_t)(kStatRows * B * sizeof(float));

  if (tid == 0) {
    s_abort = 0;
    mbar_init(&full[0], 1);
    mbar_init(&full[1], 1);
    mbar_fence_init();
  }
  __syncthreads();
  int issued[2] = {0, 0};  // copies issued per stage buffer (thread 0)
  if (tid == 0) {
    prefetch_tmap(&map);
    for (int s = 0; s < 2 && s < nst; ++s) {
      mbar_arrive_expect_tx(&full[s], box_bytes);
      tma_load_3d(stage[s], &map, p.band_lo, c, r_beg + s * kStatRows, &full[s]);
      ++issued[s];
    }
  }

  // ---- reference direction m
  if (mode == STAT_INIT) {
    if (warp == 0) {
      // first valid pixel of the partition (its line's rows) in row-major order
      long found = -1;
      const long total = (long)line.rows * ncp;
      for (long base = 0; base < total && found < 0; base += 32) {
        const long i = base + lane;
        bool ok = false;
        if (i < total) {
          const int row = line.row0 + (int)(i / ncp), col = c0 + (int)(i % ncp);
          ok = !p.mask || p.mask[(size_t)row * p.cols + col] == 0;
          if (ok) {
            const float4* px = reinterpret_cast<const float4*>(pixel_ptr(p, row, col));
            for (int f = 0; f < B4; ++f) ok = ok && finite4(__ldg(px + f));
          }
        }
        const unsigned bal = __ballot_sync(0xffffffffu, ok);
        if (bal) found = base + __ffs(bal) - 1;
      }
      if (lane == 0) s_pilot = (int)found;
    }
    __syncthreads();
    const int pi = s_pilot;
    for (int b = tid; b < B; b += kThreads) {
      float v = 0.f;
      if (pi >= 0) v = pixel_ptr(p, line.row0 + pi / ncp, c0 + pi % ncp)[b];
      s_ref[b] = v;
      if (c == c0 && chunk == 0) p.pilot[(size_t)part * B + b] = v;
    }
  } else {
    for (int b = tid; b < B; b += kThreads) s_ref[b] = p.mu0f[(size_t)part * B + b];
  }
  __syncthreads();
  if (tid == 0) {
    if (mode == STAT_INIT) {
      double n2 = 0.0;
      for (int b = 0; b < B; ++b) n2 += (double)s_ref[b] * s_ref[b];
      s_inv_ref2 = n2 > 0.0 ? (float)(1.0 / n2) : 0.f;
    } else {
      s_inv_ref2 = p.pscal[(size_t)part * PS_N + PS_INVMU2];
    }
  }
  __syncthreads();
  const float inv_ref2 = s_inv_ref2;
  const float4* ref4 = reinterpret_cast<const float4*>(s_ref);
  const bool albedo = (p.flags & MF_ALBEDO) != 0;

  // ---- SYRK ownership: 4x4 blocks of the upper triangle, blocks tid,
  // tid + 256, ...; double-float accumulators in shared memory, block-major
  // with the 32 floats (16 hi, 16 lo) of a block strided by nblk
  const int nb = BA / 4;
  const int nblk = nb * (nb + 1) / 2;
  const int bcoef = B / 4;  // block index of [a, b, 1, 0]
  float* accs = reinterpret_cast<float*>(smem_raw + L.acc_off);
  for (int q = tid; q < nblk * 32; q += kThreads) accs[q] = 0.f;

  const int e = lane & 1;
  const int slot = warp * 16 + (lane >> 1);  // 0..127
  for (int i = 0; i < nst; ++i) {
    const int sb = i & 1;
    if (!mbar_wait(&full[sb], (uint32_t)((i >> 1) & 1))) {
      if (lane == 0) atomicExch(&s_abort, 1);
    }
    __syncthreads();
    if (s_abort) break;
    // phase A: residuals e_i in place, coefficients [a, b, 1, 0]
    {
      const int row = r_beg + i * kStatRows + slot;
      const bool inb = row < r_end;
      float* px = stage[sb] + (size_t)slot * B;
      float4 x[NJ];
      const bool fin = lds_pixel<NJ>(px, inb, e, B4, x);
      const size_t pix = (size_t)(inb ? row : 0) * p.cols + c;
      const bool valid = inb && fin && (!p.mask || p.mask[pix] == 0);
      const float rho = pair_dot<NJ>(x, ref4, e, B4) * inv_ref2;
      split_residual<NJ>(x, ref4, rho, e, B4);
      if (!valid) {
#pragma unroll
        for (int j = 0; j < NJ; ++j) x[j] = make_float4(0.f, 0.f, 0.f, 0.f);
      }
      sts_pixel<NJ>(px, e, B4, x);
      if (e == 0) {
        float bcf = 0.f;
        if (mode == STAT_LITERAL && valid) {
          const float r = albedo ? rho : 1.f;
          bcf = r > 0.f ? -(r * p.alpha[pix]) : 0.f;
        }
        coef[sb][slot] = valid ? make_float4(rho - 1.f, bcf, 1.f, 0.f)
                               : make_float4(0.f, 0.f, 0.f, 0.f);
      }
    }
    __syncthreads();
    // phase B: augmented SYRK over the 128 pixels of the stage
    for (int blk = tid; blk < nblk; blk += kThreads) {
      int bi, bj;
      block_of(blk, nb, bi, bj);
      // row pointers and strides: the [a, b, 1, 0] block lives in coef[]
      const float* pa = (bi == bcoef) ? reinterpret_cast<const float*>(coef[sb]) : stage[sb] + 4 * bi;
      const float* pb = (bj == bcoef) ? reinterpret_cast<const float*>(coef[sb]) : stage[sb] + 4 * bj;
      const int sa = (bi == bcoef) ? 4 : B;
      const int sbs = (bj == bcoef) ? 4 : B;
      float hi[16], lo[16];
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        hi[q] = accs[q * nblk + blk];
        lo[q] = accs[(16 + q) * nblk + blk];
      }
      for (int s0 = 0; s0 < kStatRows; s0 += kFold) {
        float acc[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) acc[q] = 0.f;
#pragma unroll 4
        for (int s = s0; s < s0 + kFold; ++s) {
          const float4 va = *reinterpret_cast<const float4*>(pa + (size_t)s * sa);
          const float4 vb = *reinterpret_cast<const float4*>(pb + (size_t)s * sbs);
          const float a4[4] = {va.x, va.y, va.z, va.w};
          const float b4[4] = {vb.x, vb.y, vb.z, vb.w};
#pragma unroll
          for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int w = 0; w < 4; ++w) acc[u * 4 + w] = fmaf(a4[u], b4[w], acc[u * 4 + w]);
        }
#pragma unroll
        for (int q = 0; q < 16; ++q) two_sum_acc(hi[q], lo[q], acc[q]);
      }
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        accs[q * nblk + blk] = hi[q];
        accs[(16 + q) * nblk + blk] = lo[q];
      }
    }
    __syncthreads();
    if (tid == 0 && i + 2 < nst) {
      fence_proxy_async_smem();  // phase A wrote this buffer through the generic proxy
      mbar_arrive_expect_tx(&full[sb], box_bytes);
      tma_load_3d(stage[sb], &map, p.band_lo, c, r_beg + (i + 2) * kStatRows, &full[sb]);
      ++issued[sb];
    }
  }
  if (s_abort) {
    if (tid == 0) {
      // bounded wait for the last copy issued on each buffer before the CTA exits
      for (int s = 0; s < 2; ++s)
        if (issued[s] > 0) mbar_wait(&full[s], (uint32_t)((issued[s] - 1) & 1));
      p.status[part] = MF_ERR_TIMEOUT;
    }
    return;
  }

  // ---- publish this CTA's moments (double-float pairs)
  const int K1E = k1_entries(BA);
  float2* dst = p.k1part + (size_t)it.unit * K1E;
  for (int q = tid; q < nblk * 16; q += kThreads) {
    const int blk = q >> 4, w = q & 15;
    dst[q] = make_float2(accs[w * nblk + blk], accs[(16 + w) * nblk + blk]);
  }
}

#define MF_NJ_CASES(X) X(1) X(2) X(4) X(6) X(8) X(9) X(10) X(12) X(16)

cudaError_t stats_set_attributes(int nj, size_t smem) {
#define MF_CASE(NJ)                                                                    \
  case NJ:                                                                             \
    return cudaFuncSetAttribute(stats_kernel<NJ>,                                      \
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  switch (nj) { MF_NJ_CASES(MF_CASE) }
#undef MF_CASE
  return cudaErrorInvalidValue;
}

void stats_launch(int nj, int grid, size_t smem, cudaStream_t s, const CUtensorMap& map,
                  const Params& p, int mode, int pass) {
#define MF_CASE(NJ)                                                     \
  case NJ:                                                              \
    stats_kernel<NJ><<<grid, kThreads, smem, s>>>(map, p, mode, pass);  \
    return;
  switch (nj) { MF_NJ_CASES(MF_CASE) }
#undef MF_CASE
}

}  // namespace mf
