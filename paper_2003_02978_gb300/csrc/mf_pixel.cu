// Pixel kernel: the per-pixel steps of Fig. 1 (Algorithm
// AlbedoReWeightL1Filter) and the moments the next background update needs.
//
// Per valid pixel, in one read of its band window:
//   rho_i = x_i.mu0 / mu0.mu0            albedo factor, Eq. (7) (r_i = rho_i,
//                                        or 1 without albedo correction)
//   e_i   = x_i - rho_i mu0               residual of the albedo-direction split
//   p_i   = (x_i - mu^k).v = e_i.v + (rho_i - 1) mu0.v - (mu^k - mu0).v
//   init:  alpha_i^0 = p_i / (r_i q)      Eq. (3) divided by r_i (Fig. 1)
//   iter:  w_i = 1 / (alpha_i^{k-1} + eps) (Eq. (5)), pen = lambda w_i
//          alpha_i^k = max(0, (p_i - pen) / (r_i q))   (Eq. (6) with r_i, Fig. 1)
//   beta_i = r_i alpha_i^k, accumulated as sum beta, sum beta^2,
//          sum beta (rho_i - 1) and sum beta e_i (a B-vector)
// with v = (C^k)^{-1} t(mu^k) and q = t^T v prepared by the solve kernel.
//
// Layout: a CTA owns a tile of 16 adjacent detector columns over a block of
// rows; the plan sizes the row blocks so that the grid is one wave of two
// CTAs per SM (one for windows over 72 bands).  Each pipeline stage is one TMA box of 8 rows x 16 columns x
// B bands (contiguous 16 x B x 4 bytes per row in HBM), double buffered on
// full / empty mbarriers; warp w takes row w of every stage, lane pair s
// column s, so that every lane pair keeps the same column (partition) and
// its moments in registers.  The band arithmetic is packed two-wide
// (fma.rn.f32x2); alpha and the mask of the next stage are prefetched into
// registers; thread 0 refills the buffer of the previous stage at the start
// of each stage.
#include "mf_common.cuh"
#include "mf_pixel_io.cuh"
#include "mf_tma.cuh"
#include "../../include/mf.h"

namespace mf {

namespace {
constexpr int kPixThreads = kStageRows * 32;  // one warp per stage row
constexpr int kPixStages = 2;

struct PixSmem {
  size_t stage_bytes, bar_off, par_off, total;
};
// BP = 8 NJ >= B: per-column parameter stride, zero-padded so that a lane's
// band groups e + 2 j (j < NJ) load without a bounds test
__host__ __device__ inline PixSmem pix_layout(int B, int BP) {
  PixSmem L;
  L.stage_bytes = (size_t)kStageRows * kTileCols * B * sizeof(float);
  L.bar_off = kPixStages * L.stage_bytes;
  L.par_off = L.bar_off + 2 * kPixStages * sizeof(uint64_t);
  // per column: mu0f[BP], v[BP], 4 scalars
  L.total = L.par_off + (size_t)kTileCols * (2 * BP + 4) * sizeof(float);
  return L;
}
}  // namespace

// two CTAs per SM (registers capped at 128 per thread) up to 72 bands; one
// above, where the band registers would spill.  The kernel is launched
// without the programmatic attribute (measured: a pixel pass whose CTAs were
// placed early, as the solve's CTAs left, ran 4 us slower per launch); it
// still signals its dependents after its (then no-op) wait, so that the next
// solve's CTAs start their copies as the pass's CTAs finish.
constexpr int pix_ctas_per_sm(int nj) { return nj <= 9 ? 2 : 1; }

size_t pixel_smem_bytes(int B, int nj) { return pix_layout(B, 8 * nj).total + 128; }
int pixel_ctas_per_sm(int nj) { return pix_ctas_per_sm(nj); }

template <int NJ>
__global__ void __launch_bounds__(kPixThreads, pix_ctas_per_sm(NJ))
    pixel_kernel(const __grid_constant__ CUtensorMap map, Params p, int mode, int accumulate,
                 int pass) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ int s_abort;
  __shared__ int s_failed[kTileCols];
  __shared__ __align__(8) uint64_t s_never;  // fault hook: a barrier nothing arrives on

  const int li = line_of_block(p, blockIdx.x);
  const LineInfo line = p.lines[li];
  // iteration pass `pass` of a line whose iterations are done: nothing to do
  if (mode == PIX_ITER && pass > line.n_iter) return;
  accumulate = accumulate && pass < line.n_iter;
  const int local = blockIdx.x - line.blk0;
  const int ct = local % p.n_ct;
  const int rb = local / p.n_ct;
  const int c0t = ct * kTileCols;
  const int nc = min(kTileCols, p.cols - c0t);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int B = p.B, B4 = p.B4;
  constexpr int BP = 8 * NJ;
  const PixSmem L = pix_layout(B, BP);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem_raw + L.bar_off);
  uint64_t* empty = full + kPixStages;
  float* s_mu = reinterpret_cast<float*>(smem_raw + L.par_off);
  float* s_v = s_mu + kTileCols * BP;
  float* s_sc = s_v + kTileCols * BP;

  const int r_beg = line.row0 + rb * line.rb_rows;
  const int r_end = min(line.row0 + line.rows, r_beg + line.rb_rows);
  const int nst = (r_end - r_beg + kStageRows - 1) / kStageRows;
  const uint32_t box_bytes = (uint32_t)(kStageRows * kTileCols * B * sizeof(float));
  // first row of the i-th stage processed: odd passes walk the rows
  // backwards, so that a pass starts on the rows the previous pass read
  // last, which may still be in L2 (the cube is larger than L2)
  const bool backwards = (pass & 1) != 0;
  auto stage_row = [&](int i) { return r_beg + (backwards ? nst - 1 - i : i) * kStageRows; };

  if (tid == 0) {
    s_abort = 0;
    for (int q = 0; q < kPixStages; ++q) {
      mbar_init(&full[q], 1);
      mbar_init(&empty[q], kStageRows);
    }
    mbar_init(&s_never, 1);
    mbar_fence_init();
  }
  __syncthreads();
  int issued[kPixStages] = {0};  // thread 0: copies issued per stage buffer
  // every stage streamed with an evict-first L2 policy: the cube (larger
  // than L2) then does not push out what the solves re-read between passes
  // (L^-1, the moment partials, alpha); measured, this beat both the plain
  // policy (1.83 ms per retrieval) and keeping the last-read stages with an
  // evict-last policy for the next pass (1.81 ms at 3/4 of the L2) at 1.75 ms
  const uint64_t pol_stream = l2_policy_evict_first();
  auto load = [&](int q, int i) {
    mbar_arrive_expect_tx(&full[q], box_bytes);
    tma_load_3d_hint(smem_raw + q * L.stage_bytes, &map, p.band_lo, c0t, stage_row(i), &full[q],
                     pol_stream);
    ++issued[q];
  };
  if (tid == 0) {
    prefetch_tmap(&map);
    for (int i = 0; i < kPixStages && i < nst; ++i) load(i, i);
  }
  // the first stages of the cube are on their way; what follows reads the
  // previous kernel's outputs (the solve's parameters and status) and
  // writes alpha and the moments it may still read (a no-op wait, as this
  // kernel is launched in stream order)
  pdl_wait();
  pdl_trigger();
  const LaunchSpan span(p);
  // per-column parameters of the current pass
  for (int idx = tid; idx < kTileCols * BP; idx += kPixThreads) {
    const int cc = idx / BP, b = idx % BP;
    float m = 0.f, v = 0.f;
    if (cc < nc && b < B) {
      const size_t pb = (size_t)part_of(p, li, c0t + cc) * B + b;
      m = p.mu0f[pb];
      v = p.vf[pb];
    }
    s_mu[idx] = m;
    s_v[idx] = v;
  }
  if (tid < kTileCols) {
    float4 sc = make_float4(1.f, 0.f, 0.f, 0.f);
    int failed = 1;
    if (tid < nc) {
      const int part = part_of(p, li, c0t + tid);
      sc = reinterpret_cast<const float4*>(p.pscal)[part];
      failed = p.status[part] != MF_OK;
    }
    reinterpret_cast<float4*>(s_sc)[tid] = sc;
    s_failed[tid] = failed;
  }
  __syncthreads();

  const int e = lane & 1;
  const int s_col = lane >> 1;  // column within the tile
  const bool col_ok = s_col < nc;
  const int c = c0t + s_col;
  const float4 sc = reinterpret_cast<const float4*>(s_sc)[s_col];
  const float q = sc.x, muv = sc.y, coff = sc.z, invmu2 = sc.w;
  const bool failed = s_failed[s_col] != 0;
  const bool any_failed = __any_sync(0xffffffffu, failed);
  const float4* mu_s = reinterpret_cast<const float4*>(s_mu + s_col * BP) + e;
  const float4* v_s = reinterpret_cast<const float4*>(s_v + s_col * BP) + e;
  // the lane's band groups e + 2 j of a stage pixel; past the window (odd
  // B4, or a template bucket wider than B) the last group is read again:
  // mu0 and v are zero there, and those groups of the moments are dropped
  int goff[NJ];
#pragma unroll
  for (int j = 0; j < NJ; ++j) goff[j] = min(e + 2 * j, B4 - 1);
  const bool albedo = (p.flags & MF_ALBEDO) != 0;
  const bool sparse = (p.flags & MF_SPARSE) != 0;
  const bool pna = (p.flags & MF_PENALTY_NO_ALBEDO) != 0;
  const float lam = line.lambda, eps = p.eps;
  const bool iter = mode == PIX_ITER;
  const float* ain = iter ? p.alpha : p.alpha_init;

  float4 g[NJ];  // sum beta_i e_i over the lane's band groups
#pragma unroll
  for (int j = 0; j < NJ; ++j) g[j] = make_float4(0.f, 0.f, 0.f, 0.f);
  float sb = 0.f, sb2 = 0.f, sba = 0.f;
  // per-pixel terms of the objective (Eq. (8) as the shrinkage step
  // minimises it) at this pass's iterate, when the energy is asked for:
  // f_i(a) - (x_i - mu)^T C^-1 (x_i - mu) = -2 r a p + r^2 a^2 q + 2 pen r a
  const bool want_energy = p.energy != nullptr;
  float en = 0.f;

  // alpha (previous estimate or alpha_init) and the mask of stage i
  auto fetch = [&](int i, float& a_out, int& m_out) {
    const int row = stage_row(i) + warp;
    a_out = 0.f;
    m_out = 0;
    if (i < nst && row < r_end && col_ok) {
      const size_t pix = (size_t)row * p.cols + c;
      if (ain) a_out = ain[pix];
      if (p.mask) m_out = p.mask[pix];
    }
  };
  float a_nx;
  int m_nx;
  fetch(0, a_nx, m_nx);
  // fault hook (MF_FAULT=timeout): in pass 0 every warp makes one bounded
  // wait on a barrier that nothing arrives on; it runs out, and the CTA
  // leaves through the timeout path below (which first waits for the copies
  // it issued) instead of streaming its rows
  if (p.test_wait > 0 && pass == 0) {
    if (!__all_sync(0xffffffffu, mbar_wait_for(&s_never, 0, p.test_wait)) && lane == 0)
      atomicExch(&s_abort, 1);
    __syncthreads();
  }
  const int nst_run = s_abort ? 0 : nst;
  for (int i = 0; i < nst_run; ++i) {
    const int sq = i % kPixStages;
    // refill the previous stage's buffer once every warp has read it
    if (tid == 0 && i >= 1 && i - 1 + kPixStages < nst) {
      const int qr = (i - 1) % kPixStages;
      if (mbar_wait(&empty[qr], (uint32_t)(((i - 1) / kPixStages) & 1)))
        load(qr, i - 1 + kPixStages);
      else
        atomicExch(&s_abort, 1);
    }
    const float a_cur = a_nx;
    const int m_cur = m_nx;
    fetch(i + 1, a_nx, m_nx);
    // warp-uniform decision: the pair shuffles below need every lane
    if (!__all_sync(0xffffffffu, mbar_wait(&full[sq], (uint32_t)((i / kPixStages) & 1)))) {
      atomicExch(&s_abort, 1);
      break;
    }
    const int row = stage_row(i) + warp;
    const bool inb = row < r_end && col_ok;
    const float* px = reinterpret_cast<const float*>(smem_raw + sq * L.stage_bytes) +
                      (size_t)(warp * kTileCols + s_col) * B;
    float4 x[NJ];
#pragma unroll
    for (int j = 0; j < NJ; ++j) x[j] = reinterpret_cast<const float4*>(px)[goff[j]];
    // a pixel of an excluded partition is NaN when finite, 0 otherwise: an
    // exact per-element test there (its mu0 need not be finite)
    bool fin_exact = true;
    if (any_failed) {
      bool f = true;
#pragma unroll
      for (int j = 0; j < NJ; ++j) f = f && finite4(x[j]);
      fin_exact = __shfl_xor_sync(0xffffffffu, (int)f, 1) && f;
    }
    float4 ref[NJ];
#pragma unroll
    for (int j = 0; j < NJ; ++j) ref[j] = mu_s[2 * j];
    const float rho_raw = pair_dot2<NJ>(x, ref);
    // every lane's x is in registers (the dot consumed it): only now release
    // the stage to the next TMA copy, which must not overtake a pending load
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[sq]);
    const float rho = rho_raw * invmu2;
    split_residual2<NJ>(x, ref, rho);
#pragma unroll
    for (int j = 0; j < NJ; ++j) ref[j] = v_s[2 * j];
    const float pe = pair_dot2<NJ>(x, ref);

    // every band finite <=> the dot with the (finite) mu0 is finite
    const bool fin = failed ? fin_exact : isfinite(rho_raw);
    const bool valid = inb && fin && m_cur == 0;
    const float pp = pe + (rho - 1.f) * muv - coff;
    const float r = albedo ? rho : 1.f;
    float al, a_en, pen = 0.f;
    if (!iter) {
      const float a0 = p.alpha_init ? a_cur : (r > 0.f ? pp / (r * q) : 0.f);
      al = line.n_iter == 0 ? a0 : fmaxf(a0, 0.f);
      a_en = a0;  // the initial iterate is the unclamped estimate
    } else {
      const float w = sparse ? 1.f / (a_cur + eps) : 0.f;
      pen = lam * w;
      if (pna) pen = r > 0.f ? pen / r : 0.f;
      al = r > 0.f ? fmaxf((pp - pen) / (r * q), 0.f) : 0.f;
      a_en = al;
    }
    if (want_energy && e == 0 && valid && !failed && r > 0.f) {
      const float ra = r * a_en;
      en += ra * (fmaf(ra, q, -2.f * pp) + 2.f * pen);
    }
    if (!valid)
      al = 0.f;
    else if (failed)
      al = __int_as_float(0x7fc00000);
    if (inb && e == 0) {
      const size_t pix = (size_t)row * p.cols + c;
      p.alpha[pix] = al;
      if (p.ck_alpha) p.ck_alpha[(size_t)pass * p.rows * p.cols + pix] = al;
      if (!iter && p.albedo) p.albedo[pix] = valid ? r : 0.f;
    }
    if (accumulate) {
      // excluded pixels may hold non-finite bands: they add nothing
      const bool use = valid && !failed && r > 0.f;
      const float beta = use ? r * al : 0.f;
      if (e == 0) {
        sb += beta;
        sb2 = fmaf(beta, beta, sb2);
        sba = fmaf(beta, use ? rho - 1.f : 0.f, sba);
      }
      if (use) axpy2<NJ>(g, beta, x);
    }
  }
  __syncthreads();
  if (s_abort) {
    if (tid == 0) {
      // bounded wait for the last copy issued on each buffer before the CTA exits
      for (int q2 = 0; q2 < kPixStages; ++q2)
        if (issued[q2] > 0) mbar_wait(&full[q2], (uint32_t)((issued[q2] - 1) & 1));
      for (int cc = 0; cc < nc; ++cc) p.status[part_of(p, li, c0t + cc)] = MF_ERR_TIMEOUT;
    }
    return;
  }
  if (!accumulate && !want_energy) return;

  // ---- moments of the tile, per column: sum over the 8 warps (fixed
  // order); every copy has landed and been read, so the stages are free
  const int E3 = k3_entries(B);
  float* red = reinterpret_cast<float*>(smem_raw);  // [kStageRows][kTileCols][E3]
  float* mine = red + ((size_t)warp * kTileCols + s_col) * E3;
#pragma unroll
  for (int j = 0; j < NJ; ++j) {
    const int f = e + 2 * j;
    if (f < B4) {
      mine[3 + 4 * f] = g[j].x;  // offset 3: scalar stores (not 16-byte aligned)
      mine[4 + 4 * f] = g[j].y;
      mine[5 + 4 * f] = g[j].z;
      mine[6 + 4 * f] = g[j].w;
    }
  }
  if (e == 0) {
    mine[0] = sb;
    mine[1] = sb2;
    mine[2] = sba;
    mine[B + 3] = en;
  }
  __syncthreads();
  const int K3E = E3;
  for (int t = tid; t < nc * E3; t += kPixThreads) {
    const int cc = t / E3, j = t % E3;
    float sum = 0.f;
#pragma unroll
    for (int w = 0; w < kStageRows; ++w) sum += red[((size_t)w * kTileCols + cc) * E3 + j];
    const long long unit = line.k3u0 + (long long)(c0t + cc) * line.n_rb + rb;
    p.k3part[(size_t)unit * K3E + j] = sum;
  }
}

#define MF_NJ_CASES(X) X(1) X(2) X(4) X(6) X(8) X(9) X(10) X(12) X(16)

cudaError_t pixel_set_attributes(int nj, size_t smem) {
#define MF_CASE(NJ)                                                                    \
  case NJ:                                                                             \
    return cudaFuncSetAttribute(pixel_kernel<NJ>,                                      \
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  switch (nj) { MF_NJ_CASES(MF_CASE) }
#undef MF_CASE
  return cudaErrorInvalidValue;
}

void pixel_launch(int nj, int grid, size_t smem, cudaStream_t s, const CUtensorMap& map,
                  const Params& p, int mode, int accumulate, int pass) {
#define MF_CASE(NJ)                                                        \
  case NJ:                                                                 \
    launch_kernel(pixel_kernel<NJ>, grid, kPixThreads, smem, s, false, map, p, mode, accumulate, \
                  pass);                                                 \
    return;
  switch (nj) { MF_NJ_CASES(MF_CASE) }
#undef MF_CASE
}

}  // namespace mf
