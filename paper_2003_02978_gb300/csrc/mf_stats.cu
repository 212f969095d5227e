// Statistics kernel: second moments of the background of each partition.
//
// Fig. 1 (Algorithm AlbedoReWeightL1Filter) initialises mu^0 = (1/N) sum L_i
// and C^0 = (1/N) sum (L_i - mu^0)(L_i - mu^0)^T (outer product, as in
// Eq. (11)); the literal schedule recomputes C^k = (1/N) sum d_i d_i^T with
// d_i = L_i - r_i alpha_i^{k-1} t(mu^k) - mu^k at every iteration.
//
// One CTA streams one detector column over a chunk of rows: a TMA box of 128
// rows x B bands per stage, double buffered on mbarriers.  Each pixel is
// split along the partition's K reference directions q_k (pilot_dirs_kernel:
// an orthonormal basis of its first valid pixels, which spans the albedo
// direction of Sec. II-C and the strongest background modes):
//   x_i = sum_k rho_ik q_k + e_i,  rho_ik = (x_i . q_k) / (q_k . q_k),
// so that what is accumulated in float32 is small: the residual e_i and the
// centred coefficients a_ik = rho_ik - c_k.  With a covariance whose
// condition number reaches 1e7, float32 products of the unsplit pixels (or
// of a one-direction split) leave errors of 1e-4 to 1e-3 relative along the
// smallest eigenvectors; with K = 8 directions they are below 1e-6.  The CTA
// forms the augmented second moments of
//   u_i = [e_i, a_i1 .. a_iK, b_i, 1],  b_i = -r_i alpha_i^{k-1},
// a symmetric BA x BA product in 4x4 register blocks, folded every 32
// pixels into double-float (TwoSum) accumulators, and writes them out.  The
// solve kernels reduce them and assemble C exactly from
//   x_i - mu = e_i + sum_k a_ik q_k + b_i t + (sum_k c_k q_k - mu).
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
  int ncb;  // float4 groups of a pixel's coefficients [a_1 .. a_K, b, 1, 0 ..]
};
// stages | coefficients | double-float accumulators | barriers.  One
// coefficient buffer suffices: a stage's coefficients are written (phase A)
// only after the previous stage's products (phase B) are done.
__host__ __device__ inline StatSmem stat_layout(int B, int K) {
  StatSmem L;
  const int BA = aug_width(B, K);
  const int nb = BA / 4;
  const size_t nblk = (size_t)nb * (nb + 1) / 2;
  L.ncb = (BA - B) / 4;
  L.stage_bytes = (size_t)kStatRows * B * sizeof(float);
  L.stages_off = 0;
  L.coef_off = 2 * L.stage_bytes;
  L.acc_off = L.coef_off + (size_t)kStatRows * L.ncb * 4 * sizeof(float);
  L.bar_off = L.acc_off + nblk * 32 * sizeof(float);
  L.total = L.bar_off + 4 * sizeof(uint64_t);
  return L;
}
}  // namespace

size_t stats_smem_bytes(int B, int K) { return stat_layout(B, K).total + 128; }

// Reference directions of the float32 statistics split: an orthonormal basis
// q_1 .. q_K of the partition's first valid pixels (row-major over its
// columns), by modified Gram-Schmidt with one re-orthogonalisation in
// float64, rounded to float32; s_k = 1 / (q_k . q_k) of the rounded q_k and
// c_k = (q_k . m) s_k, m the mean of the pixels examined.  A pixel that adds
// no new direction (its residual below 1e-6 of its norm) is passed over; if
// fewer than K independent pixels exist the remaining q_k, s_k, c_k are 0.
// Any directions give the same moments in exact arithmetic: these keep what
// is accumulated in float32 small.  One warp per partition.
__global__ void pilot_dirs_kernel(Params p) {
  const LaunchSpan span(p);
  const int part = blockIdx.x * 4 + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (part >= p.P) return;
  const int K = p.K, B = p.B;
  const LineInfo line = p.lines[part_line(p, part)];
  const int c0 = part_col0(p, part), ncp = part_ncols(p, part);
  const long total = (long)line.rows * ncp;
  constexpr int kQ = kMaxB / 32;  // this lane's bands lane + 32 j
  double q[kMaxDirs][kQ];
  double mean[kQ];
#pragma unroll
  for (int j = 0; j < kQ; ++j) {
    mean[j] = 0.0;
#pragma unroll
    for (int k = 0; k < kMaxDirs; ++k) q[k][j] = 0.0;
  }
  auto wsum = [](double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
  };
  int n = 0, seen = 0;  // warp-uniform
  for (long base = 0; base < total && n < K; base += 32) {
    const long i = base + lane;
    bool ok = false;
    if (i < total) {
      const int row = line.row0 + (int)(i / ncp), col = c0 + (int)(i % ncp);
      ok = !p.mask || p.mask[(size_t)row * p.cols + col] == 0;
      if (ok) {
        const float4* px = reinterpret_cast<const float4*>(pixel_ptr(p, row, col));
        // every band finite (the loads are independent: no short circuit)
        for (int f = 0; f < p.B4; ++f) ok &= finite4(__ldg(px + f));
      }
    }
    unsigned bal = __ballot_sync(0xffffffffu, ok);
    while (bal && n < K) {
      const long v = base + __ffs(bal) - 1;
      bal &= bal - 1;
      const float* px = pixel_ptr(p, line.row0 + (int)(v / ncp), c0 + (int)(v % ncp));
      double x[kQ];
#pragma unroll
      for (int j = 0; j < kQ; ++j) {
        const int b = lane + 32 * j;
        x[j] = b < B ? (double)px[b] : 0.0;
        mean[j] += x[j];
      }
      ++seen;
      double xn2 = 0.0;
#pragma unroll
      for (int j = 0; j < kQ; ++j) xn2 += x[j] * x[j];
      xn2 = wsum(xn2);
      for (int pass = 0; pass < 2; ++pass)
#pragma unroll
        for (int k = 0; k < kMaxDirs; ++k) {
          if (k >= n) break;
          double d = 0.0;
#pragma unroll
          for (int j = 0; j < kQ; ++j) d += q[k][j] * x[j];
          d = wsum(d);
#pragma unroll
          for (int j = 0; j < kQ; ++j) x[j] -= d * q[k][j];
        }
      double r2 = 0.0;
#pragma unroll
      for (int j = 0; j < kQ; ++j) r2 += x[j] * x[j];
      r2 = wsum(r2);
      if (r2 > 1e-12 * xn2 && r2 > 0.0) {
        const double inv = 1.0 / sqrt(r2);
#pragma unroll
        for (int k = 0; k < kMaxDirs; ++k)
          if (k == n)
#pragma unroll
            for (int j = 0; j < kQ; ++j) q[k][j] = x[j] * inv;
        ++n;
      }
    }
  }
  const double inv_seen = seen > 0 ? 1.0 / seen : 0.0;
#pragma unroll
  for (int k = 0; k < kMaxDirs; ++k) {
    if (k >= K) break;
    double qq = 0.0, qm = 0.0;
#pragma unroll
    for (int j = 0; j < kQ; ++j) {
      const int b = lane + 32 * j;
      const float qf = (k < n && b < B) ? (float)q[k][j] : 0.f;
      if (b < B) p.pilot[((size_t)part * K + k) * B + b] = qf;
      qq += (double)qf * qf;
      qm += (double)qf * (mean[j] * inv_seen);
    }
    qq = wsum(qq);
    qm = wsum(qm);
    if (lane == 0) {
      const double sk = qq > 0.0 ? 1.0 / qq : 0.0;
      p.pilot_s[(size_t)part * K + k] = (float)sk;
      p.pilot_c[(size_t)part * K + k] = (float)(qm * sk);
    }
  }
}

void pilot_dirs_launch(cudaStream_t s, const Params& p) {
  pilot_dirs_kernel<<<(p.P + 3) / 4, 128, 0, s>>>(p);
}

static_assert(kMaxDirs + 2 <= 12, "a pixel's coefficients fill at most three float4 groups");

// Thread slot t -> 4 x 4 block (bi, bj), bi <= bj, of the upper triangle of
// nb x nb blocks, enumerated by groups of four block rows, each group column
// by column with the rows of a column fastest (column c of a group of h rows
// holds min(h, c + 1) blocks).  A warp's 32 consecutive slots then cover
// about 4 block rows x 8 block columns, so that per pixel its two float4 loads
// touch 4 + 8 distinct addresses; in row-major order they touch up to 32.
__device__ inline void tile_decode(int t, int nb, int& bi, int& bj) {
  for (int r0 = 0; r0 < nb; r0 += 4) {
    const int h = min(4, nb - r0), ncol = nb - r0;
    const int tri = h * (h + 1) / 2;  // the first h columns
    const int cnt = tri + (ncol - h) * h;
    if (t < cnt) {
      int c = 0, r;
      if (t < tri) {
        while (t >= c + 1) {
          t -= c + 1;
          ++c;
        }
        r = t;
      } else {
        c = h + (t - tri) / h;
        r = (t - tri) % h;
      }
      bi = r0 + r;
      bj = r0 + c;
      return;
    }
    t -= cnt;
  }
  bi = bj = 0;  // t >= nb (nb + 1) / 2: not reached
}

template <int NJ>
__global__ void __launch_bounds__(kThreads) stats_kernel(const __grid_constant__ CUtensorMap map,
                                                         Params p, int mode, int pass) {
  pdl_wait();
  pdl_trigger();
  const LaunchSpan span(p);
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(16) float s_dir[kMaxDirs * kMaxB];   // q_k, k < K
  __shared__ __align__(16) float s_mu0f[kMaxB];             // literal: mu^0 for r_i
  __shared__ float s_dc[kMaxDirs], s_ds[kMaxDirs];          // c_k, s_k
  __shared__ int s_abort;

  const StatItem it = stat_item(p, blockIdx.x);
  const LineInfo line = p.lines[it.line];
  // literal schedule: lines whose iterations are done take no part
  if (mode == STAT_LITERAL && pass > line.n_iter) return;
  const int c = it.c;
  const int part = part_of(p, it.line, c);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int B = p.B, B4 = p.B4, BA = p.BA, K = p.K;
  const StatSmem L = stat_layout(B, K);
  const int ncb = L.ncb;
  float* stage[2] = {reinterpret_cast<float*>(smem_raw + L.stages_off),
                     reinterpret_cast<float*>(smem_raw + L.stages_off + L.stage_bytes)};
  float4* coef = reinterpret_cast<float4*>(smem_raw + L.coef_off);
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
      // evict-first: the moment partials the solves read next stay in L2
      tma_load_3d_hint(stage[s], &map, p.band_lo, c, r_beg + s * kStatRows, &full[s],
                       l2_policy_evict_first());
      ++issued[s];
    }
  }

  // ---- the partition's reference directions (pilot_dirs_kernel), and for
  // the literal schedule mu^0 (the albedo factor of the b coefficient)
  // (one direction in the literal schedule: mu^0 with offset 1, whose
  // coefficient is the albedo factor; the solve kernel assembles likewise)
  const bool lit1 = mode == STAT_LITERAL && K == 1;
  for (int q = tid; q < K * B; q += kThreads)
    s_dir[q] = lit1 ? p.mu0f[(size_t)part * B + q] : p.pilot[(size_t)part * K * B + q];
  if (tid < K) {
    s_dc[tid] = lit1 ? 1.f : p.pilot_c[(size_t)part * K + tid];
    s_ds[tid] = lit1 ? p.pscal[(size_t)part * PS_N + PS_INVMU2] : p.pilot_s[(size_t)part * K + tid];
  }
  if (mode == STAT_LITERAL)
    for (int b = tid; b < B; b += kThreads) s_mu0f[b] = p.mu0f[(size_t)part * B + b];
  __syncthreads();
  const float inv_mu2 = mode == STAT_LITERAL ? p.pscal[(size_t)part * PS_N + PS_INVMU2] : 0.f;
  const bool albedo = (p.flags & MF_ALBEDO) != 0;

  // ---- SYRK ownership: 4x4 blocks of the upper triangle, slots tid,
  // tid + 256, ... (tile_decode); double-float accumulators in shared
  // memory, slot-major with the 32 floats (16 hi, 16 lo) of a slot strided by
  // nblk
  const int nb = BA / 4;
  const int nblk = nb * (nb + 1) / 2;
  const int bcoef = B / 4;  // first block of the coefficients
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
    // phase A: residuals e_i in place, coefficients [a_1 .. a_K, b, 1, 0 ..]
    {
      const int row = r_beg + i * kStatRows + slot;
      const bool inb = row < r_end;
      float* px = stage[sb] + (size_t)slot * B;
      float4 x[NJ];
      const bool fin = lds_pixel<NJ>(px, inb, e, B4, x);
      const size_t pix = (size_t)(inb ? row : 0) * p.cols + c;
      const bool valid = inb && fin && (!p.mask || p.mask[pix] == 0);
      float r_alb = 1.f;
      if (mode == STAT_LITERAL && albedo)
        r_alb = pair_dot2s<NJ>(x, reinterpret_cast<const float4*>(s_mu0f), e, B4) * inv_mu2;
      // coefficients on the unsplit pixel, then one subtraction per direction
      float rho[kMaxDirs];
#pragma unroll
      for (int k = 0; k < kMaxDirs; ++k)
        rho[k] = k < K ? pair_dot2s<NJ>(x, reinterpret_cast<const float4*>(s_dir + k * B), e, B4) *
                             s_ds[k]
                       : 0.f;
#pragma unroll
      for (int k = 0; k < kMaxDirs; ++k)
        if (k < K)
          split_residual2s<NJ>(x, reinterpret_cast<const float4*>(s_dir + k * B), rho[k], e, B4);
      if (!valid) {
#pragma unroll
        for (int j = 0; j < NJ; ++j) x[j] = make_float4(0.f, 0.f, 0.f, 0.f);
      }
      sts_pixel<NJ>(px, e, B4, x);
      if (e == 0) {
        float bcf = 0.f;
        if (mode == STAT_LITERAL && valid) bcf = r_alb > 0.f ? -(r_alb * p.alpha[pix]) : 0.f;
        float cf[4 * 3];
#pragma unroll
        for (int q = 0; q < 12; ++q) {
          float v = 0.f;
          if (q < K) v = rho[q] - s_dc[q];
          else if (q == K) v = bcf;
          else if (q == K + 1) v = 1.f;
          cf[q] = valid ? v : 0.f;
        }
#pragma unroll
        for (int g = 0; g < 3; ++g)
          if (g < ncb)
            coef[slot * ncb + g] = make_float4(cf[4 * g], cf[4 * g + 1], cf[4 * g + 2], cf[4 * g + 3]);
      }
    }
    __syncthreads();
    // phase B: augmented SYRK over the 128 pixels of the stage
    for (int blk = tid; blk < nblk; blk += kThreads) {
      int bi, bj;
      tile_decode(blk, nb, bi, bj);
      // row pointers and strides: the coefficient blocks live in coef[]
      const float* cbase = reinterpret_cast<const float*>(coef);
      const float* pa = (bi >= bcoef) ? cbase + 4 * (bi - bcoef) : stage[sb] + 4 * bi;
      const float* pb = (bj >= bcoef) ? cbase + 4 * (bj - bcoef) : stage[sb] + 4 * bj;
      const int sa = (bi >= bcoef) ? 4 * ncb : B;
      const int sbs = (bj >= bcoef) ? 4 * ncb : B;
      float hi[16], lo[16];
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        hi[q] = accs[q * nblk + blk];
        lo[q] = accs[(16 + q) * nblk + blk];
      }
      for (int s0 = 0; s0 < kStatRows; s0 += kFold) {
        // the 4 x 4 products on the packed f32x2 pipe (fma.rn.f32x2, each
        // element rounded as fmaf would): acc2[2 u + h] holds entries
        // (u, 2 h) and (u, 2 h + 1)
        float2 acc2[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) acc2[q] = make_float2(0.f, 0.f);
#pragma unroll 4
        for (int s = s0; s < s0 + kFold; ++s) {
          const float4 va = *reinterpret_cast<const float4*>(pa + (size_t)s * sa);
          const float4 vb = *reinterpret_cast<const float4*>(pb + (size_t)s * sbs);
          const float a4[4] = {va.x, va.y, va.z, va.w};
          const float2 b01 = make_float2(vb.x, vb.y), b23 = make_float2(vb.z, vb.w);
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const float2 au = make_float2(a4[u], a4[u]);
            acc2[2 * u] = __ffma2_rn(au, b01, acc2[2 * u]);
            acc2[2 * u + 1] = __ffma2_rn(au, b23, acc2[2 * u + 1]);
          }
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          two_sum_acc(hi[2 * q], lo[2 * q], acc2[q].x);
          two_sum_acc(hi[2 * q + 1], lo[2 * q + 1], acc2[q].y);
        }
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
      tma_load_3d_hint(stage[sb], &map, p.band_lo, c, r_beg + (i + 2) * kStatRows, &full[sb],
                       l2_policy_evict_first());
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

  // ---- publish this CTA's moments (double-float pairs), blocks in
  // row-major order of the upper triangle: block (bi, bj) at
  // bi nb - bi (bi - 1) / 2 + bj - bi
  const int K1E = k1_entries(BA);
  float2* dst = p.k1part + (size_t)it.unit * K1E;
  for (int q = tid; q < nblk * 16; q += kThreads) {
    const int slot = q >> 4, w = q & 15;
    int bi, bj;
    tile_decode(slot, nb, bi, bj);
    const int blk = bi * nb - bi * (bi - 1) / 2 + (bj - bi);
    dst[(size_t)blk * 16 + w] = make_float2(accs[w * nblk + slot], accs[(16 + w) * nblk + slot]);
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
    launch_kernel(stats_kernel<NJ>, grid, kThreads, smem, s, p.pdl != 0, map, p, mode, pass); \
    return;
  switch (nj) { MF_NJ_CASES(MF_CASE) }
#undef MF_CASE
}

}  // namespace mf
