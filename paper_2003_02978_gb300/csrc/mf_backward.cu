// Backward pass of a retrieval (the differentiation form): the hand-written
// adjoint of the unrolled procedure of Fig. 1, given the adjoint of the
// output alpha^n; gradients with respect to the unit absorption spectrum s,
// the weight multiplier lambda and (optionally) the radiance cube.
//
// The forward pass checkpoints alpha^k of every pass and, per partition and
// pass, mu^k, t^k, v^k, g^k, q^k, mean(beta)^k, var(beta)^k.  Stage k of the
// backward (k = n .. 0; stage 0 is the initialisation with beta = 0 and no
// penalty) reverses, per partition,
//   alpha^k = max(a, 0), a = (p - pen) / (r q), p = (x - mu^k).v^k,
//   q = t^k.v^k, v^k = (C^k)^{-1} t^k, C^k = (1/N) sum d d^T,
//   d_i = x_i - beta_i t^k - mu^k, t^k = mu^k (.) s,
//   mu^k = mu^0 - mean(beta) t^{k-1}, beta_i = r_i alpha^{k-1}_i,
//   w_i = 1 / (alpha^{k-1}_i + eps), pen = lambda w (or lambda w / r),
// in two passes over the cube:
//   pass A:  abar_i (the clamp's subgradient is 0 at the kink), pbar_i =
//            abar_i / (r_i q); sums P = sum pbar, X_p = sum pbar x,
//            qbar = -sum abar a / q and the lambda adjoint;
//   solve:   vbar = X_p - P mu^k + qbar t^k, zbar = (C^k)^{-1} vbar (Woodbury
//            through C^0's inverse factor, as the forward), tbar += zbar;
//   pass B:  with e1 = v.d_i = p_i - beta_i q and e2 = zbar.d_i,
//            dbar_i = -(zbar e1 + v e2) / N (the covariance adjoint is the
//            rank-2 matrix -(zbar v^T + v zbar^T)/2, so no B x B product per
//            pixel), betabar_i = (e1 zbar.t + e2 q) / N, the adjoint of
//            alpha^{k-1} = r betabar - w^2 wbar, rbar accumulations, the
//            per-pixel coefficients of the cube gradient (v^k and zbar^k);
//   post:    tbar, mubar^k, sbar += tbar (.) mu^k, mubar^0 += mubar^k, the
//            mean(beta) adjoint -mubar^k.t^{k-1} (spread as a per-partition
//            constant to the next stage) and the t^{k-1} carry.
// After stage 0: mubar^0 += sum rbar_i (x_i - 2 r_i mu^0) / |mu^0|^2 (the
// albedo factor, Eq. (7)); the cube gradient
//   xbar_i = sum_k (cv_ik v^k + cz_ik zbar^k) + rbar_i mu^0 / |mu^0|^2
//            + mubar^0 / N
// is written in one pass, and sbar, lambar are summed over the partitions.
// Pixel arithmetic follows the forward pixel kernel (albedo-direction split
// of x along mu0f, packed f32x2 band arithmetic); partition-level arithmetic
// is double-float.
#include "mf_common.cuh"
#include "mf_df.cuh"
#include "mf_dense.cuh"
#include "mf_pixel_io.cuh"
#include "mf_tma.cuh"
#include "../../include/mf.h"

namespace mf {

namespace {
constexpr int kBwThreads = kStageRows * 32;  // one warp per stage row
constexpr int kBwStages = 2;
constexpr int kBwScalars = 8;                // scalar slots of a pass's per-CTA sums

struct BwSmem {
  size_t stage_bytes, bar_off, par_off, total;
};
// per column: mu0f[BP], v[BP], zbar[BP] (zero-padded past B) and 16 scalars
__host__ __device__ inline BwSmem bw_layout(int B, int BP) {
  BwSmem L;
  L.stage_bytes = (size_t)kStageRows * kTileCols * B * sizeof(float);
  L.bar_off = kBwStages * L.stage_bytes;
  L.par_off = L.bar_off + 2 * kBwStages * sizeof(uint64_t);
  L.total = L.par_off + (size_t)kTileCols * (3 * BP + 16) * sizeof(float);
  return L;
}

__device__ __forceinline__ df ldf(const float2* q, size_t i) {
  const float2 v = q[i];
  return df{v.x, v.y};
}
__device__ __forceinline__ void stf(float2* q, size_t i, df v) { q[i] = make_float2(v.hi, v.lo); }

// sum of per-CTA partials of partition `part` (units of a pixel pass), one
// entry per thread, double-float, fixed order
__device__ df reduce_units(const Params& p, int part, const float* parts, int E, int j) {
  const LineInfo& line = p.lines[0];
  const int nunits = part_ncols(p, part) * line.n_rb;
  const float* P0 = parts + (size_t)(line.k3u0 + (long long)part_col0(p, part) * line.n_rb) * E;
  df s{0.f, 0.f};
  for (int u = 0; u < nunits; ++u) s = df_addf(s, P0[(size_t)u * E + j]);
  return s;
}

__device__ df block_sum(df v, df* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
    v = df_add(v, df{__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)});
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  df s = red[0];
  for (int i = 1; i < kWarps; ++i) s = df_add(s, red[i]);
  __syncthreads();
  return s;
}
__device__ df block_dot(const df* a, const df* b, int n, df* red) {
  df s{0.f, 0.f};
  for (int i = threadIdx.x; i < n; i += kThreads) s = df_fma(a[i], b[i], s);
  return block_sum(s, red);
}

}  // namespace

size_t bwd_pixel_smem_bytes(int B, int nj) { return bw_layout(B, 8 * nj).total + 128; }
size_t bwd_solve_smem_bytes(int B) { return ((size_t)B * linv_ld(B) + 20 * (size_t)B) * sizeof(df) + 64; }

// ---------------------------------------------------------------- pre(k)
// per-partition float scalars and v^k of stage k for the pixel passes
__global__ void __launch_bounds__(kThreads) bwd_pre_kernel(Params p, BwdParams b, int k) {
  __shared__ df red[kWarps];
  const int part = blockIdx.x, tid = threadIdx.x, B = p.B;
  const float2* cv = p.ck_vec + ((size_t)part * p.ck_stages + k) * 4 * B;
  const float* mf = p.mu0f + (size_t)part * B;
  df muv{0.f, 0.f}, coff{0.f, 0.f}, m2{0.f, 0.f};
  for (int j = tid; j < B; j += kThreads) {
    const df v = ldf(cv, CKV_V * B + j);
    const df muk = ldf(cv, CKV_MU * B + j);
    b.vkf[(size_t)part * B + j] = df_to_float(v);
    muv = df_fma(df{mf[j], 0.f}, v, muv);
    coff = df_fma(df_sub(muk, df{mf[j], 0.f}), v, coff);
    m2 = df_fma(df{mf[j], 0.f}, df{mf[j], 0.f}, m2);
  }
  muv = block_sum(muv, red);
  coff = block_sum(coff, red);
  m2 = block_sum(m2, red);
  if (tid == 0) {
    double* ps = b.psc + (size_t)part * kPsc;
    ps[PSC_Q] = p.ck_sc[((size_t)part * p.ck_stages + k) * 4 + CKS_Q];
    ps[PSC_BBAR] = p.ck_sc[((size_t)part * p.ck_stages + k) * 4 + CKS_BBAR];
    ps[PSC_MUV] = df_to_double(muv);
    ps[PSC_COFF] = df_to_double(coff);
    ps[PSC_INVM2] = 1.0 / (double)df_to_float(m2);
    ps[PSC_N] = p.dscal[(size_t)part * 4 + DS_N];
  }
}

// ------------------------------------------------------------ pixel passes
// two CTAs per SM (16 warps to hide the per-pixel latency) while the
// register cap that implies costs few spills (NJ <= 9); one above
constexpr int bw_ctas_per_sm(int nj) { return nj <= 9 ? 2 : 1; }

template <int NJ>
__global__ void __launch_bounds__(kBwThreads, bw_ctas_per_sm(NJ))
    bwd_pixel_kernel(const __grid_constant__ CUtensorMap map, Params p, BwdParams b, int k,
                     int phase) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ int s_abort;
  __shared__ int s_skip[kTileCols];

  const LineInfo line = p.lines[0];
  const int ct = blockIdx.x % p.n_ct;
  const int rb = blockIdx.x / p.n_ct;
  const int c0t = ct * kTileCols;
  const int nc = min(kTileCols, p.cols - c0t);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int B = p.B, B4 = p.B4;
  constexpr int BP = 8 * NJ;
  const BwSmem L = bw_layout(B, BP);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem_raw + L.bar_off);
  uint64_t* empty = full + kBwStages;
  float* s_mu = reinterpret_cast<float*>(smem_raw + L.par_off);
  float* s_v = s_mu + kTileCols * BP;
  float* s_z = s_v + kTileCols * BP;
  float* s_sc = s_z + kTileCols * BP;  // [kTileCols][16]

  const int r_beg = rb * line.rb_rows;
  const int r_end = min(line.rows, r_beg + line.rb_rows);
  const int nst = (r_end - r_beg + kStageRows - 1) / kStageRows;
  const uint32_t box_bytes = (uint32_t)(kStageRows * kTileCols * B * sizeof(float));
  // pass B walks the rows backwards, so that it starts on the rows pass A
  // read last (kept in L2 with an evict-last policy); the next stage's pass
  // A then starts on the rows pass B read last
  const bool backwards = phase == 1;
  auto stage_row = [&](int i) { return r_beg + (backwards ? nst - 1 - i : i) * kStageRows; };
  const int n_keep = (int)(p.l2_keep * (float)nst);
  const uint64_t pol_keep = l2_policy_evict_last(), pol_stream = l2_policy_evict_first();
  const int n = b.n_iter;
  const int S = p.ck_stages;
  const size_t npix = (size_t)p.rows * p.cols;

  if (tid == 0) {
    s_abort = 0;
    for (int q = 0; q < kBwStages; ++q) {
      mbar_init(&full[q], 1);
      mbar_init(&empty[q], kStageRows);
    }
    mbar_fence_init();
  }
  __syncthreads();
  int issued[kBwStages] = {0};
  auto load = [&](int q, int i) {
    mbar_arrive_expect_tx(&full[q], box_bytes);
    tma_load_3d_hint(smem_raw + q * L.stage_bytes, &map, p.band_lo, c0t, stage_row(i), &full[q],
                     i >= nst - n_keep ? pol_keep : pol_stream);
    ++issued[q];
  };
  if (tid == 0) {
    prefetch_tmap(&map);
    for (int i = 0; i < kBwStages && i < nst; ++i) load(i, i);
  }
  for (int idx = tid; idx < kTileCols * BP; idx += kBwThreads) {
    const int cc = idx / BP, j = idx % BP;
    float m = 0.f, v = 0.f, z = 0.f;
    if (cc < nc && j < B) {
      const int part = part_of(p, 0, c0t + cc);
      m = p.mu0f[(size_t)part * B + j];
      v = b.vkf[(size_t)part * B + j];
      if (phase == 1) z = b.zf[((size_t)part * S + k) * B + j];
    }
    s_mu[idx] = m;
    s_v[idx] = v;
    s_z[idx] = z;
  }
  if (tid < kTileCols) {
    float* sc = s_sc + tid * 16;
    int skip = 1;
    if (tid < nc) {
      const int part = part_of(p, 0, c0t + tid);
      const double* ps = b.psc + (size_t)part * kPsc;
      sc[0] = (float)ps[PSC_Q];
      sc[1] = (float)ps[PSC_MUV];
      sc[2] = (float)ps[PSC_COFF];
      sc[3] = (float)ps[PSC_INVM2];
      sc[4] = (float)ps[PSC_N];
      sc[5] = (float)ps[PSC_CNEXT];
      sc[6] = (float)ps[PSC_ZT];
      sc[7] = (float)ps[PSC_ZMU0];
      sc[8] = (float)ps[PSC_ZOFF];
      skip = p.status[part] != MF_OK;
    }
    s_skip[tid] = skip;
  }
  __syncthreads();

  const int e = lane & 1;
  const int s_col = lane >> 1;
  const bool col_ok = s_col < nc;
  const int c = c0t + s_col;
  const float* sc = s_sc + s_col * 16;
  const float q = sc[0], muv = sc[1], coff = sc[2], invm2 = sc[3], Nf = sc[4], cnext = sc[5];
  const float zt = sc[6], zmu0 = sc[7], zoff = sc[8];
  const bool skip = s_skip[s_col] != 0;
  const float4* mu_s = reinterpret_cast<const float4*>(s_mu + s_col * BP) + e;
  const float4* v_s = reinterpret_cast<const float4*>(s_v + s_col * BP) + e;
  const float4* z_s = reinterpret_cast<const float4*>(s_z + s_col * BP) + e;
  int goff[NJ];
#pragma unroll
  for (int j = 0; j < NJ; ++j) goff[j] = min(e + 2 * j, B4 - 1);
  const bool albedo = (p.flags & MF_ALBEDO) != 0;
  const bool sparse = (p.flags & MF_SPARSE) != 0;
  const bool pna = (p.flags & MF_PENALTY_NO_ALBEDO) != 0;
  const float lam = line.lambda, eps = p.eps;
  const float* a_k = p.ck_alpha + (size_t)k * npix;
  const float* a_prev = k > 0 ? p.ck_alpha + (size_t)(k - 1) * npix : nullptr;
  const float* abar_in = k == n ? b.grad_alpha : b.abar[k & 1];
  float* abar_out = k > 0 ? b.abar[(k - 1) & 1] : nullptr;

  float4 acc[NJ];
#pragma unroll
  for (int j = 0; j < NJ; ++j) acc[j] = make_float4(0.f, 0.f, 0.f, 0.f);
  float sums[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};

  for (int i = 0; i < nst; ++i) {
    const int sq = i % kBwStages;
    if (tid == 0 && i >= 1 && i - 1 + kBwStages < nst) {
      const int qr = (i - 1) % kBwStages;
      if (mbar_wait(&empty[qr], (uint32_t)(((i - 1) / kBwStages) & 1)))
        load(qr, i - 1 + kBwStages);
      else
        atomicExch(&s_abort, 1);
    }
    const int row = stage_row(i) + warp;
    const bool inb = row < r_end && col_ok;
    const size_t pix = (size_t)(line.row0 + row) * p.cols + c;
    float ak = 0.f, ap = 0.f, abin = 0.f;
    int m = 1;
    if (inb) {
      ak = a_k[pix];
      if (a_prev) ap = a_prev[pix];
      abin = abar_in[pix];
      m = p.mask ? p.mask[pix] : 0;
    }
    if (!__all_sync(0xffffffffu, mbar_wait(&full[sq], (uint32_t)((i / kBwStages) & 1)))) {
      atomicExch(&s_abort, 1);
      break;
    }
    const float* px = reinterpret_cast<const float*>(smem_raw + sq * L.stage_bytes) +
                      (size_t)(warp * kTileCols + s_col) * B;
    float4 x[NJ];
#pragma unroll
    for (int j = 0; j < NJ; ++j) x[j] = reinterpret_cast<const float4*>(px)[goff[j]];
    float4 ref[NJ];
#pragma unroll
    for (int j = 0; j < NJ; ++j) ref[j] = mu_s[2 * j];
    const float rho_raw = pair_dot2<NJ>(x, ref);
    // every lane's x is in registers (the dot consumed it): only now release
    // the stage to the next TMA copy, which must not overtake a pending load
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[sq]);
    const float rho = rho_raw * invm2;
    split_residual2<NJ>(x, ref, rho);  // x <- e = x - rho mu0f
#pragma unroll
    for (int j = 0; j < NJ; ++j) ref[j] = v_s[2 * j];
    const float pe = pair_dot2<NJ>(x, ref);
    float ze = 0.f;
    if (phase == 1) {
#pragma unroll
      for (int j = 0; j < NJ; ++j) ref[j] = z_s[2 * j];
      ze = pair_dot2<NJ>(x, ref);
    }
    const float r = albedo ? rho : 1.f;
    const bool use = inb && !skip && m == 0 && isfinite(rho_raw) && r > 0.f;
    const float pp = pe + (rho - 1.f) * muv - coff;            // (x - mu^k).v^k
    const bool pos = (k == 0 && n == 0) ? true : ak > 0.f;      // clamp's subgradient
    const float abk = abin + r * cnext;                         // adjoint of alpha^k
    const float ab = use && pos ? abk : 0.f;
    const float rq = r * q;
    const float pbar = ab / rq;
    const float penbar = -ab / rq;
    float w = 0.f, beta = 0.f, pen = 0.f;
    if (k > 0) {
      w = sparse ? 1.f / (ap + eps) : 0.f;
      beta = r * ap;
      pen = pna ? lam * w / r : lam * w;
    }
    if (phase == 0) {
      if (use) {
        axpy2<NJ>(acc, pbar, x);
        if (e == 0) {
          sums[0] += pbar;
          sums[1] = fmaf(pbar, rho, sums[1]);
          sums[2] -= ab * ak / q;
          sums[3] = fmaf(penbar, pna ? w / r : w, sums[3]);
        }
      }
    } else {
      const float zx = ze + (rho - 1.f) * zmu0 - zoff;        // zbar.(x - mu^k)
      const float e1 = pp - beta * q;                         // v^k . d_i
      const float e2 = zx - beta * zt;                        // zbar . d_i
      const float bb = (e1 * zt + e2 * q) / Nf;               // betabar_i (pass-B part)
      const float wbar = penbar * (pna ? lam / r : lam);
      float rb_add = 0.f;
      if (use) {
        rb_add = -ab * ak / r + ap * bb + ak * cnext;
        if (pna) rb_add += ab * pen / (r * rq);
        if (e == 0) {
          sums[0] = fmaf(beta, e1, sums[0]);
          sums[1] = fmaf(beta, e2, sums[1]);
          sums[2] += e1;
          sums[3] += e2;
        }
      }
      // rbar accumulated over the stages (both lanes of the pair read the
      // old value before lane 0 stores the new one)
      const float rprev = inb && k != n ? b.rbar[pix] : 0.f;
      const float rtot = rprev + rb_add;
      if (inb && e == 0) {
        if (abar_out) abar_out[pix] = use ? r * bb - w * w * wbar : 0.f;
        b.rbar[pix] = rtot;
        if (b.coef) {
          float2 cf = make_float2(0.f, 0.f);
          if (use) cf = make_float2(pbar - e2 / Nf, -e1 / Nf);
          reinterpret_cast<float2*>(b.coef)[pix * S + k] = cf;
        }
      }
      if (k == 0 && use && albedo) {
        // rbar is final: sum rbar_i x_i = (sum rbar rho) mu0f + sum rbar e
        axpy2<NJ>(acc, rtot, x);
        if (e == 0) {
          sums[4] = fmaf(rtot, rho, sums[4]);
          sums[5] = fmaf(rtot, r, sums[5]);
        }
      }
    }
  }
  __syncthreads();
  if (s_abort) {
    if (tid == 0) {
      for (int q2 = 0; q2 < kBwStages; ++q2)
        if (issued[q2] > 0) mbar_wait(&full[q2], (uint32_t)((issued[q2] - 1) & 1));
      for (int cc = 0; cc < nc; ++cc) p.status[part_of(p, 0, c0t + cc)] = MF_ERR_TIMEOUT;
    }
    return;
  }
  // per-column sums over the 8 warps (fixed order) -> partials
  const int E = bwd_entries(B);
  float* red = reinterpret_cast<float*>(smem_raw);  // [kStageRows][kTileCols][E]
  float* mine = red + ((size_t)warp * kTileCols + s_col) * E;
#pragma unroll
  for (int j = 0; j < NJ; ++j) {
    const int f = e + 2 * j;
    if (f < B4) {
      mine[kBwScalars + 4 * f] = acc[j].x;
      mine[kBwScalars + 4 * f + 1] = acc[j].y;
      mine[kBwScalars + 4 * f + 2] = acc[j].z;
      mine[kBwScalars + 4 * f + 3] = acc[j].w;
    }
  }
  if (e == 0)
    for (int j = 0; j < kBwScalars; ++j) mine[j] = j < 6 ? sums[j] : 0.f;
  __syncthreads();
  for (int t = tid; t < nc * E; t += kBwThreads) {
    const int cc = t / E, j = t % E;
    float sum = 0.f;
#pragma unroll
    for (int w2 = 0; w2 < kStageRows; ++w2) sum += red[((size_t)w2 * kTileCols + cc) * E + j];
    const long long unit = line.k3u0 + (long long)(c0t + cc) * line.n_rb + rb;
    b.bpart[(size_t)unit * E + j] = sum;
  }
}

// ------------------------------------------------------------ solve(k)
// vbar from the pass-A sums; zbar = (C^k)^{-1} vbar
namespace {
// Y = L^{-1} U, Z = L^{-T} Y for nr right-hand sides (columns of U, B each),
// L^{-1} row-major lower (diagonal included) in X; compensated dots
}  // namespace

__global__ void __launch_bounds__(kThreads, 4) bwd_solve_kernel(Params p, BwdParams b, int k) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ df red[kWarps];
  __shared__ df s_sc[8];
  __shared__ df s_W[16];
  __shared__ df s_c[3];
  __shared__ int s_bad;
  __shared__ __align__(8) uint64_t s_xbar;
  const int part = blockIdx.x, tid = threadIdx.x, B = p.B;
  const int S = p.ck_stages;
  const size_t pb = (size_t)part * B;
  double* ps = b.psc + (size_t)part * kPsc;
  if (p.status[part] != MF_OK) {
    for (int j = tid; j < B; j += kThreads) b.zf[((size_t)part * S + k) * B + j] = 0.f;
    if (tid == 0) ps[PSC_ZT] = ps[PSC_ZMU0] = ps[PSC_ZOFF] = ps[PSC_PSUM] = ps[PSC_QBAR] = 0.0;
    return;
  }
  df* X = reinterpret_cast<df*>(smem_raw);  // L^{-1} (packed rows), later the direct path's matrix
  float4* UP0 = reinterpret_cast<float4*>(X + (size_t)B * linv_ld(B));  // (vbar, g) interleaved
  float4* UP1 = UP0 + B;                                               // (t^k, d) interleaved
  float4* YP0 = UP1 + B;
  float4* YP1 = YP0 + B;
  df* vb = reinterpret_cast<df*>(YP1 + B);   // vbar
  df* G = vb + B;
  df* T = G + B;                             // t^k
  df* D = T + B;                             // t^{k-1} - t^k
  df* Y0 = D + B;
  df* Y1 = Y0 + B;
  df* Y2 = Y1 + B;
  df* Y3 = Y2 + B;
  df* Z0 = Y3 + B;
  df* Z1 = Z0 + B;
  df* Z2 = Z1 + B;
  df* Z3 = Z2 + B;
  const int E = bwd_entries(B);
  // L^{-1} of the partition into shared memory by one bulk copy, in flight
  // during the reductions below
  if (tid == 0) {
    const size_t n = linv_packed(B);
    const uint32_t bytes = (uint32_t)(n * sizeof(float2));
    mbar_init(&s_xbar, 1);
    mbar_fence_init();
    mbar_arrive_expect_tx(&s_xbar, bytes);
    bulk_load(X, p.Linv + (size_t)part * n, bytes, &s_xbar);
  }
  if (tid < 4) s_sc[tid] = reduce_units(p, part, b.bpart, E, tid);
  const float2* cv = p.ck_vec + ((size_t)part * S + k) * 4 * B;
  __syncthreads();
  const df Psum = s_sc[0], Prho = s_sc[1], Sq = s_sc[2], Slam = s_sc[3];
  for (int j = tid; j < B; j += kThreads) {
    const df V = reduce_units(p, part, b.bpart, E, kBwScalars + j);
    const df mf{p.mu0f[pb + j], 0.f};
    const df muk = ldf(cv, CKV_MU * B + j);
    const df tk = ldf(cv, CKV_T * B + j);
    df x = df_fma(Prho, mf, V);                     // sum pbar x
    x = df_sub(x, df_mul(Psum, muk));
    vb[j] = df_fma(Sq, tk, x);
    T[j] = tk;
    G[j] = ldf(cv, CKV_G * B + j);
    D[j] = k > 0 ? df_sub(ldf(cv - 4 * B, CKV_T * B + j), tk) : df{0.f, 0.f};
    UP0[j] = pack_pair(vb[j], G[j]);
    UP1[j] = pack_pair(T[j], D[j]);
  }
  __syncthreads();
  if (!__syncthreads_and(mbar_wait(&s_xbar, 0))) {
    // the copy did not complete in time (uniform decision): record it, give
    // the copy a second bounded wait and leave
    if (tid == 0) p.status[part] = MF_ERR_TIMEOUT;
    mbar_wait(&s_xbar, 0);
    return;
  }
  df* zb = Z0;
  if (k == 0) {
    const float4* U[1] = {UP0};  // (vbar, g = 0)
    float4* Yv[1] = {YP0};
    df* Zv[2] = {Z0, Z1};
    c0inv_apply<1>(X, B, U, Yv, Zv);
  } else {
    const float4* U[2] = {UP0, UP1};
    float4* Yv[2] = {YP0, YP1};
    df* Zv[4] = {Z0, Z1, Z2, Z3};
    c0inv_apply<2>(X, B, U, Yv, Zv);
    // W = U^T C0^{-1} U (3 x 3, U = [g, t, d]) and U^T C0^{-1} vbar
    const df* ua[12] = {G, G, G, T, T, T, D, D, D, G, T, D};
    const df* zv[12] = {Z1, Z2, Z3, Z1, Z2, Z3, Z1, Z2, Z3, Z0, Z0, Z0};
    for (int t = 0; t < 12; ++t) {
      const df v = block_dot(ua[t], zv[t], B, red);
      if (tid == 0) s_W[t] = v;
    }
    __syncthreads();
    if (tid == 0) {
      const double* ck = p.ck_sc + ((size_t)part * S + k) * 4;
      const df bbar = df_from_double(ck[CKS_BBAR]), var = df_from_double(ck[CKS_VAR]);
      const df zero{0.f, 0.f}, one{1.f, 0.f}, m1{-1.f, 0.f};
      const df mb2 = df_mul(bbar, bbar);
      // M = [[0, -1, 0], [-1, var, 0], [0, 0, mean(beta)^2]]
      df M[9] = {zero, m1, zero, m1, var, zero, zero, zero, mb2};
      df A3[9], rhs[3];
      for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 3; ++j) {
          df a = i == j ? one : zero;
          for (int l = 0; l < 3; ++l) a = df_fma(M[i * 3 + l], s_W[l * 3 + j], a);
          A3[i * 3 + j] = a;
        }
        df r = zero;
        for (int l = 0; l < 3; ++l) r = df_fma(M[i * 3 + l], s_W[9 + l], r);
        rhs[i] = r;
      }
      // Cramer's rule, with the Hadamard-ratio test of the forward
      auto cof = [&](int i, int j) {
        const int r0 = (i + 1) % 3, r1 = (i + 2) % 3, c0 = (j + 1) % 3, c1 = (j + 2) % 3;
        return df_sub(df_mul(A3[r0 * 3 + c0], A3[r1 * 3 + c1]), df_mul(A3[r0 * 3 + c1], A3[r1 * 3 + c0]));
      };
      df det = zero;
      for (int j = 0; j < 3; ++j) det = df_fma(A3[j], cof(0, j), det);
      float hr = 1.f;
      for (int i = 0; i < 3; ++i) {
        float n2 = 0.f;
        for (int j = 0; j < 3; ++j) n2 = fmaf(A3[i * 3 + j].hi, A3[i * 3 + j].hi, n2);
        hr *= sqrtf(n2);
      }
      hr = fabsf(det.hi) / fmaxf(hr, 1e-30f);
      s_bad = (!df_isfinite(det) || det.hi == 0.f || hr < 1e-8f) ? 1 : 0;
      if (!s_bad) {
        const df id = df_recip(det);
        for (int i = 0; i < 3; ++i) {
          df num = zero;
          for (int j = 0; j < 3; ++j) num = df_fma(cof(j, i), rhs[j], num);
          s_c[i] = df_mul(num, id);
        }
      }
    }
    __syncthreads();
    if (s_bad) {
      // direct: C^k = C^0 + U M U^T assembled from C^0 (float64) and
      // factorised (as the forward's fallback)
      const double* Sg = p.S + (size_t)part * B * B;
      const double* ck = p.ck_sc + ((size_t)part * S + k) * 4;
      const df bbar = df_from_double(ck[CKS_BBAR]), var = df_from_double(ck[CKS_VAR]);
      const df mb2 = df_mul(bbar, bbar);
      const DfMat Xm{reinterpret_cast<float*>(X), B, B * B};
      for (int idx = tid; idx < B * B; idx += kThreads) {
        const int i = idx / B, j = idx % B;
        if (j < i) continue;
        df c = df_from_double(Sg[idx]);
        c = df_sub(c, df_add(df_mul(G[i], T[j]), df_mul(T[i], G[j])));
        c = df_fma(var, df_mul(T[i], T[j]), c);
        c = df_fma(mb2, df_mul(D[i], D[j]), c);
        Xm.set(i, j, c);
      }
      const bool ok = chol_inv_df(Xm, B, Y1);  // Y1 holds 1/diag(U)
      if (ok) xtx_apply_df(Xm, B, Y1, vb, Y2, Z0);
      if (!ok) {
        if (tid == 0) p.status[part] = MF_ERR_NOT_SPD;
        for (int j = tid; j < B; j += kThreads) Z0[j] = df{0.f, 0.f};
        __syncthreads();
      }
    } else {
      const df c0 = s_c[0], c1 = s_c[1], c2 = s_c[2];
      for (int j = tid; j < B; j += kThreads) {
        df zc = df_mul(Z1[j], c0);
        zc = df_fma(Z2[j], c1, zc);
        zc = df_fma(Z3[j], c2, zc);
        Z0[j] = df_sub(Z0[j], zc);
      }
      __syncthreads();
    }
  }
  // zbar and its dot products
  df* mfv = Y0;  // mu0f as double-float
  df* dmu = Y1;  // mu^k - mu0f
  for (int j = tid; j < B; j += kThreads) {
    b.zf[((size_t)part * S + k) * B + j] = df_to_float(zb[j]);
    mfv[j] = df{p.mu0f[pb + j], 0.f};
    dmu[j] = df_sub(ldf(cv, CKV_MU * B + j), mfv[j]);
  }
  __syncthreads();
  const df zt = block_dot(zb, T, B, red);
  const df zm = block_dot(zb, mfv, B, red);
  const df zo = block_dot(zb, dmu, B, red);
  if (tid == 0) {
    ps[PSC_ZT] = df_to_double(zt);
    ps[PSC_ZMU0] = df_to_double(zm);
    ps[PSC_ZOFF] = df_to_double(zo);
    ps[PSC_PSUM] = df_to_double(Psum);
    ps[PSC_QBAR] = df_to_double(Sq);
    b.lbar[part] += df_to_double(Slam);
  }
}

// ------------------------------------------------------------- post(k)
__global__ void __launch_bounds__(kThreads) bwd_post_kernel(Params p, BwdParams b, int k) {
  __shared__ df red[kWarps];
  __shared__ df s_sc[6];
  const int part = blockIdx.x, tid = threadIdx.x, B = p.B;
  const int S = p.ck_stages;
  const size_t pb = (size_t)part * B;
  double* ps = b.psc + (size_t)part * kPsc;
  if (p.status[part] != MF_OK) {
    if (tid == 0) ps[PSC_CNEXT] = 0.0;
    return;
  }
  const int E = bwd_entries(B);
  if (tid < 6) s_sc[tid] = reduce_units(p, part, b.bpart, E, tid);
  __syncthreads();
  const df S1 = s_sc[0], S2 = s_sc[1], S3 = s_sc[2], S4 = s_sc[3], Srrho = s_sc[4], Srr = s_sc[5];
  const df N = df_from_double(ps[PSC_N]);
  const df invN = df_recip(N);
  const df Psum = df_from_double(ps[PSC_PSUM]), Sq = df_from_double(ps[PSC_QBAR]);
  const float2* cv = p.ck_vec + ((size_t)part * S + k) * 4 * B;
  const double bbar_k = p.ck_sc[((size_t)part * S + k) * 4 + CKS_BBAR];
  const bool albedo = (p.flags & MF_ALBEDO) != 0;
  df bmb{0.f, 0.f};  // dot of mubar^k with t^{k-1}
  df m2{0.f, 0.f};
  for (int j = tid; j < B; j += kThreads) {
    const df v = ldf(cv, CKV_V * B + j);
    const df tk = ldf(cv, CKV_T * B + j);
    const df muk = ldf(cv, CKV_MU * B + j);
    const df z{b.zf[((size_t)part * S + k) * B + j], 0.f};
    df tb = df_fma(Sq, v, z);
    tb = df_add(tb, ldf(b.carry, pb + j));
    tb = df_fma(df_fma(z, S1, df_mul(v, S2)), invN, tb);
    df mb = df_mul(df{-1.f, 0.f}, df_mul(Psum, v));
    mb = df_fma(df_fma(z, S3, df_mul(v, S4)), invN, mb);
    mb = df_add(mb, df_mulf(tb, p.k[j]));
    b.sbar[pb + j] += df_to_double(df_mul(tb, muk));
    df m0b = df_add(ldf(b.mubar0, pb + j), mb);
    if (k > 0) {
      const df tprev = ldf(cv - 4 * B, CKV_T * B + j);
      bmb = df_fma(mb, tprev, bmb);
      stf(b.carry, pb + j, df_mul(df_from_double(-bbar_k), mb));
    }
    stf(b.mubar0, pb + j, m0b);
    const df mu0 = ldf(p.mu0, pb + j);
    m2 = df_fma(mu0, mu0, m2);
  }
  bmb = block_sum(bmb, red);
  m2 = block_sum(m2, red);
  if (k > 0) {
    if (tid == 0) ps[PSC_CNEXT] = -df_to_double(df_mul(bmb, invN));
    return;
  }
  // stage 0: the albedo factor's adjoint, then mubar^0 / N for the cube gradient
  const df im2 = df_recip(m2);
  for (int j = tid; j < B; j += kThreads) {
    df m0b = ldf(b.mubar0, pb + j);
    if (albedo) {
      const df mu0 = ldf(p.mu0, pb + j);
      const df mf{p.mu0f[pb + j], 0.f};
      const df VR = reduce_units(p, part, b.bpart, E, kBwScalars + j);
      df rx = df_fma(Srrho, mf, VR);                       // sum rbar_i x_i
      rx = df_sub(rx, df_mul(df_mul(df{2.f, 0.f}, Srr), mu0));
      m0b = df_fma(rx, im2, m0b);
    }
    stf(b.mubar0, pb + j, m0b);
    b.mu0bar_n[pb + j] = df_to_float(df_mul(m0b, invN));
  }
  if (tid == 0) {
    ps[PSC_CNEXT] = 0.0;
    ps[PSC_INVM2] = df_to_double(im2);
  }
}

// ------------------------------------------------------------ cube gradient
// xbar_i = sum_k (cv_ik v^k + cz_ik zbar^k) + rbar_i mu^0 / |mu^0|^2 + mubar^0 / N
// for valid pixels of partitions that did not fail; 0 elsewhere.  One CTA
// per (column, block of rows); a lane pair per pixel.
template <int NJ>
__global__ void __launch_bounds__(kThreads) bwd_cube_kernel(Params p, BwdParams b, int rows_per) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int c = blockIdx.x % p.cols;
  const int blk = blockIdx.x / p.cols;
  const int part = part_of(p, 0, c);
  const int B = p.B, B4 = p.B4, S = p.ck_stages;
  constexpr int BP = 8 * NJ;
  float* sV = reinterpret_cast<float*>(smem_raw);  // [S][BP]
  float* sZ = sV + (size_t)S * BP;                  // [S][BP]
  float* sM = sZ + (size_t)S * BP;                  // mu^0 * rbar scale (albedo), [BP]
  float* sN = sM + BP;                              // mubar^0 / N, [BP]
  float* sF = sN + BP;                              // mu0f, [BP]
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const bool failed = p.status[part] != MF_OK;
  const double im2 = b.psc[(size_t)part * kPsc + PSC_INVM2];
  const bool albedo = (p.flags & MF_ALBEDO) != 0;
  for (int idx = tid; idx < S * BP; idx += kThreads) {
    const int kk = idx / BP, j = idx % BP;
    float v = 0.f, z = 0.f;
    if (j < B) {
      v = df_to_float(ldf(p.ck_vec + ((size_t)part * S + kk) * 4 * B, CKV_V * B + j));
      z = b.zf[((size_t)part * S + kk) * B + j];
    }
    sV[idx] = v;
    sZ[idx] = z;
  }
  for (int j = tid; j < BP; j += kThreads) {
    const bool in = j < B;
    sM[j] = in && albedo ? (float)(df_to_double(ldf(p.mu0, (size_t)part * B + j)) * im2) : 0.f;
    sN[j] = in ? b.mu0bar_n[(size_t)part * B + j] : 0.f;
    sF[j] = in ? p.mu0f[(size_t)part * B + j] : 0.f;
  }
  __syncthreads();
  const int e = lane & 1;
  const int slot = warp * 16 + (lane >> 1);
  const int r0 = blk * rows_per;
  const int r1 = min(p.rows, r0 + rows_per);
  for (int row = r0 + slot; row < r1 + 128; row += kThreads / 2) {
    if (__all_sync(0xffffffffu, row >= r1)) break;
    const bool inb = row < r1;
    const size_t pix = (size_t)row * p.cols + c;
    float4 acc[NJ];
#pragma unroll
    for (int j = 0; j < NJ; ++j) acc[j] = make_float4(0.f, 0.f, 0.f, 0.f);
    // validity as in the forward: not masked, dot with mu0f finite
    float d = 0.f;
    if (inb && !failed) {
      const float4* px = reinterpret_cast<const float4*>(pixel_ptr(p, row, c));
      for (int f = e; f < B4; f += 2) {
        const float4 x = px[f];
        const float4 m = reinterpret_cast<const float4*>(sF)[f];
        d = fmaf(x.x, m.x, fmaf(x.y, m.y, fmaf(x.z, m.z, fmaf(x.w, m.w, d))));
      }
    }
    d += __shfl_xor_sync(0xffffffffu, d, 1);
    const bool valid = inb && !failed && isfinite(d) && (!p.mask || p.mask[pix] == 0);
    if (valid) {
      const float2* cf = reinterpret_cast<const float2*>(b.coef) + pix * S;
      for (int kk = 0; kk < S; ++kk) {
        const float2 w = cf[kk];
        const float4* V4 = reinterpret_cast<const float4*>(sV + (size_t)kk * BP) + e;
        const float4* Z4 = reinterpret_cast<const float4*>(sZ + (size_t)kk * BP) + e;
#pragma unroll
        for (int j = 0; j < NJ; ++j) {
          const float4 v = V4[2 * j], z = Z4[2 * j];
          acc[j].x = fmaf(w.x, v.x, fmaf(w.y, z.x, acc[j].x));
          acc[j].y = fmaf(w.x, v.y, fmaf(w.y, z.y, acc[j].y));
          acc[j].z = fmaf(w.x, v.z, fmaf(w.y, z.z, acc[j].z));
          acc[j].w = fmaf(w.x, v.w, fmaf(w.y, z.w, acc[j].w));
        }
      }
      const float rb = b.rbar[pix];
      const float4* M4 = reinterpret_cast<const float4*>(sM) + e;
      const float4* N4 = reinterpret_cast<const float4*>(sN) + e;
#pragma unroll
      for (int j = 0; j < NJ; ++j) {
        const float4 m = M4[2 * j], nn = N4[2 * j];
        acc[j].x = fmaf(rb, m.x, acc[j].x + nn.x);
        acc[j].y = fmaf(rb, m.y, acc[j].y + nn.y);
        acc[j].z = fmaf(rb, m.z, acc[j].z + nn.z);
        acc[j].w = fmaf(rb, m.w, acc[j].w + nn.w);
      }
    }
    if (inb) {
      float4* out = reinterpret_cast<float4*>(b.grad_cube + pix * B);
#pragma unroll
      for (int j = 0; j < NJ; ++j) {
        const int f = e + 2 * j;
        if (f < B4) out[f] = acc[j];
      }
    }
  }
}

// ------------------------------------------------------- final reduction
__global__ void __launch_bounds__(kThreads) bwd_final_kernel(Params p, BwdParams b) {
  __shared__ double red[kThreads];
  const int tid = threadIdx.x, B = p.B;
  for (int j = tid; j < B; j += kThreads) {
    double s = 0.0;
    for (int part = 0; part < p.P; ++part)
      if (p.status[part] == MF_OK) s += b.sbar[(size_t)part * B + j];
    b.grad_k[j] = (float)s;
  }
  double l = 0.0;
  for (int part = tid; part < p.P; part += kThreads)
    if (p.status[part] == MF_OK) l += b.lbar[part];
  red[tid] = l;
  __syncthreads();
  for (int o = kThreads / 2; o > 0; o >>= 1) {
    if (tid < o) red[tid] += red[tid + o];
    __syncthreads();
  }
  if (tid == 0) *b.grad_lambda = (float)red[0];
}

#define MF_BW_NJ_CASES(X) X(1) X(2) X(4) X(6) X(8) X(9) X(10) X(12) X(16)

cudaError_t bwd_set_attributes(int nj, size_t smem_pixel, size_t smem_solve) {
  cudaError_t e = cudaErrorInvalidValue;
#define MF_CASE(NJ)                                                                       \
  case NJ:                                                                                \
    e = cudaFuncSetAttribute(bwd_pixel_kernel<NJ>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                             (int)smem_pixel);                                            \
    break;
  switch (nj) { MF_BW_NJ_CASES(MF_CASE) }
#undef MF_CASE
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(bwd_solve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)smem_solve);
}

void bwd_launch_stage(int nj, int grid_pixel, size_t smem_pixel, size_t smem_solve,
                      cudaStream_t s, const CUtensorMap& map, const Params& p,
                      const BwdParams& b, int k) {
  bwd_pre_kernel<<<p.P, kThreads, 0, s>>>(p, b, k);
#define MF_CASE(NJ)                                                                 \
  case NJ:                                                                          \
    bwd_pixel_kernel<NJ><<<grid_pixel, kBwThreads, smem_pixel, s>>>(map, p, b, k, 0); \
    bwd_solve_kernel<<<p.P, kThreads, smem_solve, s>>>(p, b, k);                    \
    bwd_pixel_kernel<NJ><<<grid_pixel, kBwThreads, smem_pixel, s>>>(map, p, b, k, 1); \
    break;
  switch (nj) { MF_BW_NJ_CASES(MF_CASE) }
#undef MF_CASE
  bwd_post_kernel<<<p.P, kThreads, 0, s>>>(p, b, k);
}

void bwd_launch_final(int nj, size_t, cudaStream_t s, const Params& p, const BwdParams& b) {
  if (b.grad_cube) {
    const int rows_per = 512;
    const int nblk = (p.rows + rows_per - 1) / rows_per;
    const size_t smem = ((size_t)(2 * p.ck_stages + 3) * 8 * nj) * sizeof(float);
#define MF_CASE(NJ)                                                                    \
  case NJ:                                                                             \
    bwd_cube_kernel<NJ><<<p.cols * nblk, kThreads, smem, s>>>(p, b, rows_per);          \
    break;
    switch (nj) { MF_BW_NJ_CASES(MF_CASE) }
#undef MF_CASE
  }
  bwd_final_kernel<<<1, kThreads, 0, s>>>(p, b);
}

}  // namespace mf
