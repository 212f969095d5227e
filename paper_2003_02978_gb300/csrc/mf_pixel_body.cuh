// Pixel pass, one CTA's work (pixel_block): the per-pixel steps of Fig. 1 (Algorithm
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
#pragma once
#include "mf_common.cuh"
#include "mf_pixel_io.cuh"
#include "mf_tma.cuh"
#include "../../include/mf.h"

namespace mf {

constexpr int kPixThreads = kStageRows * 32;  // one warp per stage row
constexpr int kPixStages = 2;

struct PixSmem {
  size_t stage_bytes, par_off, total;
};
// BP = 8 NJ >= B: per-column parameter stride, zero-padded so that a lane's
// band groups e + 2 j (j < NJ) load without a bounds test
__host__ __device__ inline PixSmem pix_layout(int B, int BP) {
  PixSmem L;
  L.stage_bytes = (size_t)kStageRows * kTileCols * B * sizeof(float);
  L.par_off = kPixStages * L.stage_bytes;
  // per column: mu0f[BP], v[BP], 4 scalars
  L.total = L.par_off + (size_t)kTileCols * (2 * BP + 4) * sizeof(float);
  return L;
}

// two CTAs per SM (registers capped at 128 per thread) up to 72 bands; one
// above, where the band registers would spill
constexpr int pix_ctas_per_sm(int nj) { return nj <= 9 ? 2 : 1; }

// a pixel CTA's mbarriers: full[kPixStages], empty[kPixStages], the fault
// hook's; and the phases each has completed
constexpr int kPixBars = 2 * kPixStages + 1;
struct PixPhases {
  uint32_t full[kPixStages], empty[kPixStages];
};
// a[q] by selects, without a run-time index into a local array
__device__ __forceinline__ uint32_t pick_phase(const uint32_t (&a)[kPixStages], int q) {
  uint32_t v = a[0];
#pragma unroll
  for (int j = 1; j < kPixStages; ++j) v = q == j ? a[j] : v;
  return v;
}
__device__ __forceinline__ void pixel_bars_init(uint64_t* bars) {
  for (int q = 0; q < kPixStages; ++q) {
    mbar_init(&bars[q], 1);
    mbar_init(&bars[kPixStages + q], kStageRows);
  }
  mbar_init(&bars[2 * kPixStages], 1);
  mbar_fence_init();
}

// One pixel CTA's work: row block x column tile `blk` of pass `pass`.
// bars: the CTA's mbarriers, initialised by the caller (pixel_bars_init);
// ph: the phases they completed before this call, advanced here.  ready()
// is called by every thread once the first cube stages are on their way and
// before anything written by another kernel or work item is read; false
// sends the CTA down the timeout path.  Returns false after a timeout (the
// tile's partitions are marked MF_ERR_TIMEOUT and every copy the call issued
// has landed), true otherwise.  kQueue: called from the persistent
// work-queue kernel (no timeline span of its own).
template <int NJ, bool kQueue, class Ready>
__device__ __forceinline__ bool pixel_block(const CUtensorMap& map, const Params& p, int mode,
                                            int accumulate, int pass, int blk,
                                            unsigned char* smem_raw, uint64_t* bars,
                                            PixPhases& ph, Ready&& ready) {
  __shared__ int s_abort;
  __shared__ int s_failed[kTileCols];

  const int li = line_of_block(p, blk);
  const LineInfo line = p.lines[li];
  // iteration pass `pass` of a line whose iterations are done: nothing to do
  if (mode == PIX_ITER && pass > line.n_iter) return true;
  accumulate = accumulate && pass < line.n_iter;
  const int local = blk - line.blk0;
  const int ct = local % p.n_ct;
  const int rb = local / p.n_ct;
  const int c0t = ct * kTileCols;
  const int nc = min(kTileCols, p.cols - c0t);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int B = p.B, B4 = p.B4;
  constexpr int BP = 8 * NJ;
  const PixSmem L = pix_layout(B, BP);
  uint64_t* full = bars;
  uint64_t* empty = bars + kPixStages;
  uint64_t* never = bars + 2 * kPixStages;  // fault hook: a barrier nothing arrives on
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

  if (tid == 0) s_abort = 0;
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
  // the first stages of the cube are on their way; what follows reads what
  // the solves wrote (the per-column parameters and status) and writes alpha
  // and the moments they may still read: ready() waits for them (the
  // per-pass kernel: a no-op programmatic wait, as it is launched in stream
  // order; the work queue: the solves of the tile's partitions)
  const bool go = ready();
  if (!go && tid == 0) s_abort = 1;
  const LaunchSpan span(p, !kQueue);
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
    if (!__all_sync(0xffffffffu, mbar_wait_for(never, 0, p.test_wait)) && lane == 0)
      atomicExch(&s_abort, 1);
    __syncthreads();
  }
  const int nst_run = s_abort ? 0 : nst;
  for (int i = 0; i < nst_run; ++i) {
    const int sq = i % kPixStages;
    // refill the previous stage's buffer once every warp has read it
    if (tid == 0 && i >= 1 && i - 1 + kPixStages < nst) {
      const int qr = (i - 1) % kPixStages;
      if (mbar_wait(&empty[qr], (uint32_t)((pick_phase(ph.empty, qr) + (i - 1) / kPixStages) & 1)))
        load(qr, i - 1 + kPixStages);
      else
        atomicExch(&s_abort, 1);
    }
    const float a_cur = a_nx;
    const int m_cur = m_nx;
    fetch(i + 1, a_nx, m_nx);
    // warp-uniform decision: the pair shuffles below need every lane
    if (!__all_sync(0xffffffffu,
                    mbar_wait(&full[sq], (uint32_t)((pick_phase(ph.full, sq) + i / kPixStages) & 1)))) {
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
        if (issued[q2] > 0)
          mbar_wait(&full[q2], (uint32_t)((pick_phase(ph.full, q2) + issued[q2] - 1) & 1));
      for (int cc = 0; cc < nc; ++cc) p.status[part_of(p, li, c0t + cc)] = MF_ERR_TIMEOUT;
    }
    return false;
  }
  // every stage was loaded once and released once: one phase of its full
  // and of its empty barrier each
  // (the work queue keeps ph in shared memory: one thread updates it, and
  // the queue's next barrier publishes it)
  if (!kQueue || tid == 0) {
#pragma unroll
    for (int q2 = 0; q2 < kPixStages; ++q2) {
      const uint32_t n = nst > q2 ? (uint32_t)((nst - q2 + kPixStages - 1) / kPixStages) : 0u;
      ph.full[q2] += n;
      ph.empty[q2] += n;
    }
  }
  if (!accumulate && !want_energy) return true;

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
  return true;
}

}  // namespace mf
