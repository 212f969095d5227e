// Solve work of one partition (bodies of the solve kernels and of the
// persistent work queue): the small dense linear algebra of the background model, one
// CTA per partition, all in double-float arithmetic (mf_df.cuh).
//
// solve_init (after the initial statistics pass; Fig. 1 initialisation):
//   reduce the per-CTA augmented moments, assemble mu^0 and
//   C^0 = (1/N) sum (x_i - mu^0)(x_i - mu^0)^T exactly from them, factorise
//   C^0 = L L^T (blocked Cholesky, L^{-1} formed in the same sweep), and
//   solve C^0 v = t^0 with t^0 = mu^0 (.) s (Eq. (9)); q = t^T v is the
//   normaliser of Eq. (3).
// solve_iter (after each pixel pass; Fig. 1 loop body, Eqs. (10)-(11)):
//   mu^{k+1} = mu^0 - mean(beta) t^k and, with t = t^{k+1},
//   d = t^k - t^{k+1} and g = mean(beta (x - mu^0)),
//   C^{k+1} = C^0 - (g t^T + t g^T) + mean(beta)^2 d d^T + var(beta) t t^T
//           = C^0 + U M U^T,  U = [g, t, d],
//   an exact expansion of Eq. (11).  v = (C^{k+1})^{-1} t follows from C^0's
//   inverse factor by the Woodbury identity:
//   v = z_t - Z (I + M W)^{-1} M W e_2,  Z = C0^{-1} U,  W = U^T Z,
//   with C0^{-1} d = C0^{-1} t^k - C0^{-1} t^{k+1} reusing the previous z_t.
//   det(C^{k+1}) = det(C^0) det(I + M W) > 0 is checked (positive definite).
// solve_literal (literal schedule, Fig. 1 as printed): assemble C^k from a
//   fresh statistics pass over d_i, factorise and solve, every iteration.
#pragma once
#include "mf_common.cuh"
#include "mf_df.cuh"
#include "mf_dense.cuh"
#include "mf_tma.cuh"
#include "../../include/mf.h"

namespace mf {

namespace {

__device__ __forceinline__ df ldf(const float2* p, size_t i) {
  const float2 v = p[i];
  return df{v.x, v.y};
}
__device__ __forceinline__ void stf(float2* p, size_t i, df v) { p[i] = make_float2(v.hi, v.lo); }

__device__ __forceinline__ df shfl_df(df v, int src) {
  return df{__shfl_sync(0xffffffffu, v.hi, src), __shfl_sync(0xffffffffu, v.lo, src)};
}

// CTA-wide double-float sum, fixed order; every thread gets the result
__device__ df block_sum_df(df v, df* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = df_add(v, df_shfl_xor(v, o));
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  df s = red[0];
  for (int i = 1; i < kWarps; ++i) s = df_add(s, red[i]);
  return s;
}

// dot product of length n by one warp (lanes stride the index), all lanes
// get the result
__device__ __forceinline__ df warp_dot_df(const df* a, const df* b, int n) {
  Dot2 d;
  for (int i = threadIdx.x & 31; i < n; i += 32) d.add(a[i], b[i]);
  df v = d.result();
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = df_add(v, df_shfl_xor(v, o));
  return v;
}

// several dots at once: dot t (t < nd) = a[t] . b[t], one warp per dot,
// written to out[t]; one barrier
__device__ void multi_dot_df(const df* const* a, const df* const* b, int nd, int n, df* out) {
  const int w = threadIdx.x >> 5;
  for (int t = w; t < nd; t += kWarps) {
    const df v = warp_dot_df(a[t], b[t], n);
    if ((threadIdx.x & 31) == 0) out[t] = v;
  }
  __syncthreads();
}

__device__ df block_dot_df(const df* a, const df* b, int n, df* red) {
  Dot2 d;
  for (int i = threadIdx.x; i < n; i += kThreads) d.add(a[i], b[i]);
  return block_sum_df(d.result(), red);
}

// bulk prefetch of `bytes` (a multiple of 16) at `src` (16-byte aligned)
// into L2; no completion to wait for
__device__ __forceinline__ void prefetch_l2_bulk(const void* src, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}

// While a solve kernel runs, the HBM would otherwise idle: at its start
// (before its dependency wait: the cube is read-only), prefetch into L2 the
// first p.pf_stages stages (8 rows of a 16-column tile each) of every CTA of
// the pixel pass `pass` that follows, in that pass's row order, so that the
// pass finds them there.  Items (pixel CTA, stage) are spread over the
// solve's CTAs; threads 0-7 take a stage's rows, one bulk prefetch of the
// tile's contiguous row segment each.  Single-line plans only.  Measured on
// the flightline: 4 stages (45 MB per pass) take 12 us off the pixel passes
// of a retrieval and cost the solves 2 us; deeper prefetch, or prefetch
// issued after the wait, slows the solves more than it helps the passes.
__device__ void prefetch_pixel_pass(const Params& p, int pass) {
  if (p.pf_stages <= 0 || p.n_lines != 1 || threadIdx.x >= kStageRows) return;
  const LineInfo& line = p.line0;
  const bool backwards = (pass & 1) != 0;
  const int items = p.n_blocks * p.pf_stages;
  for (int w = blockIdx.x; w < items; w += gridDim.x) {
    const int b = w % p.n_blocks, i = w / p.n_blocks;
    const int local = b - line.blk0;
    const int ct = local % p.n_ct, rb = local / p.n_ct;
    const int c0t = ct * kTileCols, nc = min(kTileCols, p.cols - c0t);
    const int r_beg = line.row0 + rb * line.rb_rows;
    const int r_end = min(line.row0 + line.rows, r_beg + line.rb_rows);
    const int nst = (r_end - r_beg + kStageRows - 1) / kStageRows;
    if (i >= nst) continue;
    const int r = r_beg + (backwards ? nst - 1 - i : i) * kStageRows + threadIdx.x;
    if (r < r_end)
      prefetch_l2_bulk(p.cube + ((size_t)r * p.cols + c0t) * p.bands_total,
                       (uint32_t)(nc * p.bands_total * sizeof(float)));
  }
}

// reduce the per-CTA augmented moments of `part` into the full symmetric
// BA x BA matrix A; each thread keeps 2 x 8 loads in flight
__device__ void reduce_k1(const Params& p, int part, const DfMat& A) {
  const int BA = p.BA, K1E = k1_entries(BA), nb = BA / 4;
  const LineInfo& line = p.lines[part_line(p, part)];
  const int nunits = part_ncols(p, part) * line.n_sc;
  const float2* P0 = p.k1part + (size_t)(line.k1u0 + (long long)part_col0(p, part) * line.n_sc) * K1E;
  constexpr int kU = 8;
  if (p.k1_colmajor) {
    // units of Q (column-major floats, BA x BA, BA a multiple of 4): R = the
    // sum of the units' Q into A, two entries per load, four entries x four
    // units = 16 loads in flight per thread; then G = R + R^T in place
    constexpr int kH = 4, kUq = 4;
    const float2* Q0 = P0;
    const size_t ustride = K1E;  // float2 per unit
    const int BB = BA * BA, BB2 = BB / 2;
    for (int q0 = threadIdx.x; q0 < BB2; q0 += kH * kThreads) {
      df sx[kH], sy[kH];
#pragma unroll
      for (int h = 0; h < kH; ++h) sx[h] = sy[h] = df{0.f, 0.f};
      for (int u0 = 0; u0 < nunits; u0 += kUq) {
        float2 v[kH][kUq];
#pragma unroll
        for (int h = 0; h < kH; ++h)
#pragma unroll
          for (int k = 0; k < kUq; ++k) {
            const int q = q0 + h * kThreads, u = u0 + k;
            v[h][k] = (q < BB2 && u < nunits) ? Q0[(size_t)u * ustride + q] : make_float2(0.f, 0.f);
          }
#pragma unroll
        for (int h = 0; h < kH; ++h)
#pragma unroll
          for (int k = 0; k < kUq; ++k) {
            sx[h] = df_addf(sx[h], v[h][k].x);
            sy[h] = df_addf(sy[h], v[h][k].y);
          }
      }
#pragma unroll
      for (int h = 0; h < kH; ++h) {
        const int q = 2 * (q0 + h * kThreads);  // Q_mj at j BA + m
        if (q < BB) {
          A.set(q % BA, q / BA, sx[h]);
          A.set((q + 1) % BA, (q + 1) / BA, sy[h]);
        }
      }
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < BB; idx += kThreads) {
      const int a = idx / BA, b = idx - a * BA;
      if (a > b) continue;
      const df g = df_add(A.get(a, b), A.get(b, a));
      A.set(a, b, g);
      A.set(b, a, g);
    }
    __syncthreads();
    return;
  }
  for (int q0 = threadIdx.x; q0 < K1E; q0 += 2 * kThreads) {
    df sum[2] = {df{0.f, 0.f}, df{0.f, 0.f}};
    for (int u0 = 0; u0 < nunits; u0 += kU) {
      float2 v[2][kU];
#pragma unroll
      for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int k = 0; k < kU; ++k) {
          const int q = q0 + h * kThreads, u = u0 + k;
          v[h][k] = (q < K1E && u < nunits) ? P0[(size_t)u * K1E + q] : make_float2(0.f, 0.f);
        }
#pragma unroll
      for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int k = 0; k < kU; ++k) sum[h] = df_add(sum[h], df{v[h][k].x, v[h][k].y});
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int q = q0 + h * kThreads;
      if (q >= K1E) continue;
      int bi, bj;
      tri_decode(q >> 4, nb, bi, bj);
      const int w = q & 15;
      const int i = 4 * bi + (w >> 2), j = 4 * bj + (w & 3);
      A.set(i, j, sum[h]);
      A.set(j, i, sum[h]);
    }
  }
  __syncthreads();
}

// C = (1/N) sum (e + sum_k a_k q_k + b u_b + u_1)(...)^T from the augmented
// moments G of [e, a_1 .. a_K, b, 1] (symmetric in A; coefficient column c
// at row / column B + c, c < W = K + 2), written into the upper triangle
// (diagonal included) of A's leading B x B block; the border rows B.. of A
// are read, not written.  The coefficient vectors are T_c = q_c (c < K,
// float, K x B in Q), T_K = u_b (null: zero, the initial statistics) and
// T_{K+1} = u_1.  With
//   P_ic = G_ic + sum_d G_cd T_id,
//   C_ij N = G_ij + sum_c (T_jc P_ic + T_ic G_jc),
// the same sum of terms as expanding the outer product.  scratch: W B
// double-floats.
__device__ void assemble(const Params& p, const DfMat& A, const float* Q, const df* ub,
                         const df* u1, df invN, double* S_out, df* scratch) {
  const int B = p.B, K = p.K, W = K + 2;
  const int tid = threadIdx.x;
  auto T = [&](int c, int i) -> df {
    if (c < K) return df{Q[c * B + i], 0.f};
    return c == K ? ub[i] : u1[i];
  };
  df* P = scratch;
  for (int idx = tid; idx < W * B; idx += kThreads) {
    const int c = idx / B, i = idx - c * B;
    if (c == K && !ub) continue;
    df v = A.get(B + c, i);
    for (int d = 0; d < W; ++d) {
      if (d == K && !ub) continue;
      v = df_fma(A.get(B + c, B + d), T(d, i), v);
    }
    P[idx] = v;
  }
  __syncthreads();
  // the upper triangle's entries (row j, column i >= j, row-major) spread
  // evenly over the block
  const int ntri = B * (B + 1) / 2;
  for (int t = tid; t < ntri; t += kThreads) {
    int j, i;
    tri_decode(t, B, j, i);
    df v = A.get(j, i);  // G_ji = G_ij
    for (int c = 0; c < W; ++c) {
      if (c == K && !ub) continue;
      v = df_fma(T(c, j), P[c * B + i], v);
      v = df_fma(T(c, i), A.get(B + c, j), v);
    }
    v = df_mul(v, invN);
    A.set(j, i, v);
    if (S_out) {
      const double d = df_to_double(v);
      S_out[(size_t)i * B + j] = d;
      S_out[(size_t)j * B + i] = d;
    }
  }
  __syncthreads();
}

// The partition's directions q_k into shared memory (Q, K x B floats) and
// w = sum_k c_k q_k, and from the reduced moments the mean
//   mu = w + (sum_i e_i + sum_k (sum_i a_ik) q_k) / N;
// u1 = w - mu (the constant column of the initial statistics).
__device__ void init_mean(const Params& p, int part, const DfMat& A, df invN, float* Q, df* mu,
                          df* u1) {
  const int B = p.B, K = p.K, cc = B + K + 1;
  for (int q = threadIdx.x; q < K * B; q += kThreads) Q[q] = p.pilot[(size_t)part * K * B + q];
  __syncthreads();
  for (int b = threadIdx.x; b < B; b += kThreads) {
    df w{0.f, 0.f}, sa = A.get(b, cc);
    for (int k = 0; k < K; ++k) {
      const df qk{Q[k * B + b], 0.f};
      w = df_fma(df{p.pilot_c[(size_t)part * K + k], 0.f}, qk, w);
      sa = df_fma(A.get(B + k, cc), qk, sa);
    }
    mu[b] = df_add(w, df_mul(sa, invN));
    u1[b] = df_sub(w, mu[b]);
  }
  __syncthreads();
}

__device__ void fail_partition(const Params& p, int part, bool init) {
  const int B = p.B;
  const size_t pb = (size_t)part * B;
  for (int b = threadIdx.x; b < B; b += kThreads) {
    p.vf[pb + b] = 0.f;
    if (init) {
      p.mu0f[pb + b] = 0.f;
      stf(p.mu0, pb + b, df{0.f, 0.f});
      stf(p.tprev, pb + b, df{0.f, 0.f});
      stf(p.zt, pb + b, df{0.f, 0.f});
    }
  }
  if (threadIdx.x == 0) {
    p.status[part] = MF_ERR_NOT_SPD;
    reinterpret_cast<float4*>(p.pscal)[part] = make_float4(1.f, 0.f, 0.f, 0.f);
  }
  if (p.energy)
    for (int k = threadIdx.x; k < p.energy_stride; k += kThreads)
      p.energy[(size_t)part * p.energy_stride + k] = __longlong_as_double(0x7ff8000000000000LL);
}

// Fig. 1 initialisation of partition `part` (see the top of this file);
// smem_raw holds solve_init_smem_bytes.  Reads only what the statistics
// pass wrote.  kQueue: called from the persistent work-queue kernel, where a
// concurrent work item's timeout may change the status word: it is read
// once for the whole CTA.
template <bool kQueue>
__device__ __forceinline__ void solve_init_part(const Params& p, int part,
                                                unsigned char* smem_raw) {
  const int tid = threadIdx.x;
  const int B = p.B, BA = p.BA, K = p.K;
  const size_t pb = (size_t)part * B;
  const DfMat A{reinterpret_cast<float*>(smem_raw), BA, BA * BA};
  df* vmu = reinterpret_cast<df*>(smem_raw) + (size_t)BA * BA;  // mu^0
  df* vu3 = vmu + B;             // sum c_k q_k - mu^0, later mu^0 - mu0f
  df* vt = vu3 + B;              // t^0
  df* vy = vt + B;
  df* vz = vy + B;
  df* invd = vz + B;
  df* vmf = invd + B;            // mu0f
  df* scr = vmf + B;             // (K + 2) B: assemble's scratch
  float* vq = reinterpret_cast<float*>(scr + (size_t)(K + 2) * B);  // directions, K x B
  const bool stat_failed =
      kQueue ? __syncthreads_or(p.status[part] != MF_OK) != 0 : p.status[part] != MF_OK;
  if (stat_failed) return;  // the statistics pass timed out
  if (p.fault_notspd) {  // fault hook (MF_FAULT=notspd)
    fail_partition(p, part, true);
    return;
  }

  reduce_k1(p, part, A);
  const df N = A.get(B + K + 1, B + K + 1);
  const bool enough = N.hi > (float)B;
  const df invN = enough ? df_recip(N) : df{0.f, 0.f};
  init_mean(p, part, A, invN, vq, vmu, vu3);
  assemble(p, A, vq, nullptr, vu3, invN, p.S + (size_t)part * B * B, scr);
  const bool ok = enough && chol_inv_df(A, B, invd);
  if (!ok) {
    fail_partition(p, part, true);
    return;
  }
  for (int b = tid; b < B; b += kThreads) {
    vt[b] = df_mulf(vmu[b], p.k[b]);
    const float mf = df_to_float(vmu[b]);
    vmf[b] = df{mf, 0.f};
    vu3[b] = df_sub(vmu[b], vmf[b]);
  }
  __syncthreads();
  xtx_apply_df(A, B, invd, vt, vy, vz);  // z = (C^0)^{-1} t
  __shared__ df s_d4[4];
  {
    const df* da[4] = {vt, vmf, vu3, vmf};
    const df* db[4] = {vz, vz, vz, vmf};
    multi_dot_df(da, db, 4, B, s_d4);
  }
  const df q = s_d4[0], muv = s_d4[1], coff = s_d4[2], n2 = s_d4[3];
  // store L^{-1} (packed rows: linv_row), mean, target, solution
  const size_t xn = linv_packed(B);
  float2* X = p.Linv + (size_t)part * xn;
  for (int idx = tid; idx < (int)xn; idx += kThreads) {
    int i = (int)((sqrtf(8.f * (float)idx + 1.f) - 1.f) * 0.5f);  // row: linv_row(i) <= idx
    if (linv_row(i) > idx) --i;
    else if (linv_row(i + 1) <= idx) ++i;
    const int j = idx - linv_row(i);
    stf(X, idx, j < i ? A.get(i, j) : invd[i]);
  }
  for (int b = tid; b < B; b += kThreads) {
    stf(p.mu0, pb + b, vmu[b]);
    p.mu0f[pb + b] = vmf[b].hi;
    p.vf[pb + b] = df_to_float(vz[b]);
    stf(p.zt, pb + b, vz[b]);
    stf(p.tprev, pb + b, vt[b]);
    stf(p.muk, pb + b, vmu[b]);
  }
  if (p.ck_vec) {  // checkpoint of stage 0 for the backward pass
    float2* cv = p.ck_vec + (size_t)part * p.ck_stages * 4 * B;
    for (int b = tid; b < B; b += kThreads) {
      stf(cv, CKV_MU * B + b, vmu[b]);
      stf(cv, CKV_T * B + b, vt[b]);
      stf(cv, CKV_V * B + b, vz[b]);
      stf(cv, CKV_G * B + b, df{0.f, 0.f});
    }
    if (tid == 0) {
      double* cs = p.ck_sc + (size_t)part * p.ck_stages * 4;
      cs[CKS_Q] = df_to_double(q);
      cs[CKS_BBAR] = 0.0;
      cs[CKS_VAR] = 0.0;
    }
  }
  if (tid == 0) {
    const bool good = q.hi > 0.f && df_isfinite(q);
    reinterpret_cast<float4*>(p.pscal)[part] =
        make_float4(df_to_float(q), df_to_float(muv), df_to_float(coff),
                    1.0f / df_to_float(n2));
    double* ds = p.dscal + (size_t)part * 4;
    ds[DS_N] = df_to_double(N);
    // objective at the initial iterate: sum_i (x_i - mu^0)^T (C^0)^-1 (x_i - mu^0)
    // = N tr((C^0)^-1 C^0) = N B; the pixel pass adds its per-pixel terms
    if (p.energy) p.energy[(size_t)part * p.energy_stride] = df_to_double(N) * (double)B;
    ds[DS_BBAR] = 0.0;
    ds[DS_Q] = df_to_double(q);
    ds[DS_N2] = df_to_double(n2);
    p.status[part] = good ? MF_OK : MF_ERR_NOT_SPD;
  }
}

// Fig. 1 loop body for partition `part` after pixel pass `pass` - 1 (see the
// top of this file); smem_raw holds solve_iter_smem_bytes.  xbar: the
// mbarrier of the L^-1 copy and ph_x its completed phases, advanced here.
// Per-pass kernel (kQueue false): xbar is initialised here, and the reads of
// data two or more launches back start before the programmatic wait.  Work
// queue (kQueue): xbar was initialised once by the caller; ready() is the
// dependency wait (the previous pass's pixel items over the partition's
// columns) and comes before any read.  Returns false after a timed-out copy
// (status MF_ERR_TIMEOUT) or wait, true otherwise.
template <bool kQueue, class Ready>
__device__ __forceinline__ bool solve_iter_part(const Params& p, int mode, int pass, int part,
                                                unsigned char* smem_raw, uint64_t* xbar,
                                                uint32_t& ph_x, Ready&& ready) {
  __shared__ df s_y[3];
  __shared__ int s_bad;
  const int tid = threadIdx.x;
  const int B = p.B;
  const size_t pb = (size_t)part * B;
  if (pass > p.lines[part_line(p, part)].n_iter) return true;  // the line's iterations are done
  if constexpr (kQueue) {
    if (!ready()) return false;
  }
  // L^{-1} (packed rows, linv_row), later the direct path's B x B matrix
  df* X = reinterpret_cast<df*>(smem_raw);
  float4* UP = reinterpret_cast<float4*>(X + (size_t)B * linv_ld(B));  // (g, t^{k+1}) interleaved
  float4* YP = UP + B;
  df* mom = reinterpret_cast<df*>(YP + B);  // B + 3 moments (padded to B + 8)
  df* U0 = mom + B + 8;                     // g
  df* U1 = U0 + B;                          // t^{k+1}
  df* U2 = U1 + B;                          // t^k - t^{k+1}
  df* Y0 = U2 + B;
  df* Y1 = Y0 + B;
  df* Z0 = Y1 + B;
  df* Z1 = Z0 + B;
  df* Z2 = Z1 + B;
  df* vmf = Z2 + B;
  df* vmk = vmf + B;
  df* vv = vmk + B;

  // this thread's band b = tid (B <= kThreads): the partition's vectors,
  // loaded before the moment reduction so that their latency overlaps it
  const int b = tid;
  df mu0{0.f, 0.f}, tk{0.f, 0.f}, ztk{0.f, 0.f};
  float mu0f = 0.f, kb = 0.f;
  if (b < B) {
    mu0 = ldf(p.mu0, pb + b);
    tk = ldf(p.tprev, pb + b);
    ztk = ldf(p.zt, pb + b);
    mu0f = p.mu0f[pb + b];
    kb = p.k[b];
  }
  const double* ds = p.dscal + (size_t)part * 4;
  const double Nd = ds[DS_N];
  // L^{-1} of the partition into shared memory by one bulk copy, in flight
  // during the moment reduction
  const bool solve = mode != SOLVE_MEAN_ONLY;
  if (solve && tid == 0) {
    const size_t n = linv_packed(B);
    const uint32_t bytes = (uint32_t)(n * sizeof(float2));
    if constexpr (kQueue) {
      // L^-1 was written by another work item's generic stores, the copy
      // reads it through the async proxy
      fence_proxy_async_global();
    } else {
      mbar_init(xbar, 1);
      mbar_fence_init();
    }
    mbar_arrive_expect_tx(xbar, bytes);
    bulk_load(X, p.Linv + (size_t)part * n, bytes, xbar);
  }
  const uint32_t xpar = ph_x & 1u;
  if (solve) ++ph_x;  // the copy completes one phase of xbar
  if constexpr (!kQueue) {
    // all of the above comes from kernels two or more launches back; the
    // moments, the status and every write below wait for the pixel pass
    if (mode != SOLVE_MEAN_ONLY) prefetch_pixel_pass(p, pass);
    pdl_wait();
    pdl_trigger();
  }
  const LaunchSpan span(p, !kQueue);
  const bool failed =
      kQueue ? __syncthreads_or(p.status[part] != MF_OK) != 0 : p.status[part] != MF_OK;
  if (failed) {
    // a failed partition: its copy lands before the CTA leaves
    if constexpr (kQueue) {
      return !solve || __syncthreads_and(mbar_wait(xbar, xpar));
    } else {
      if (solve && tid == 0) mbar_wait(xbar, xpar);
      return true;
    }
  }

  const int K3E = k3_entries(B);
  const LineInfo& line = p.lines[part_line(p, part)];
  const int nunits = part_ncols(p, part) * line.n_rb;
  const float* P0 = p.k3part + (size_t)(line.k3u0 + (long long)part_col0(p, part) * line.n_rb) * K3E;
  for (int t = tid; t < B + 4; t += kThreads) {
    // eight loads in flight, then their fixed-order sum
    df s{0.f, 0.f};
    int u = 0;
    for (; u + 8 <= nunits; u += 8) {
      float v[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) v[q] = P0[(size_t)(u + q) * K3E + t];
#pragma unroll
      for (int q = 0; q < 8; ++q) s = df_addf(s, v[q]);
    }
    for (; u < nunits; ++u) s = df_addf(s, P0[(size_t)u * K3E + t]);
    mom[t] = s;
  }
  __syncthreads();
  const df N = df_from_double(Nd);
  const df invN = df_recip(N);
  const df sb = mom[0], sb2 = mom[1], sba = mom[2];
  const df bbar = df_mul(sb, invN);
  const df var = df_sub(df_mul(sb2, invN), df_mul(bbar, bbar));
  if (b < B) {
    const df mf{mu0f, 0.f};
    const df mk = df_sub(mu0, df_mul(bbar, tk));
    const df t1 = df_mulf(mk, kb);
    // g = mean(beta (x - mu0)), x - mu0 = e + (rho - 1) mu0f + (mu0f - mu0)
    df g = df_fma(sba, mf, mom[3 + b]);
    g = df_fma(sb, df_sub(mf, mu0), g);
    U0[b] = df_mul(g, invN);
    U1[b] = t1;
    U2[b] = df_sub(tk, t1);
    UP[b] = pack_pair(U0[b], U1[b]);
    vmf[b] = mf;
    vmk[b] = mk;
  }
  if (mode == SOLVE_MEAN_ONLY) {
    __syncthreads();
    for (int i = tid; i < B; i += kThreads) {
      stf(p.muk, pb + i, vmk[i]);
      stf(p.tprev, pb + i, U1[i]);
    }
    if (tid == 0) p.dscal[(size_t)part * 4 + DS_BBAR] = df_to_double(bbar);
    return true;
  }
  if (!__syncthreads_and(mbar_wait(xbar, xpar))) {
    // the copy did not complete in time (uniform decision): record it, give
    // the copy a second bounded wait and leave
    if (tid == 0) p.status[part] = MF_ERR_TIMEOUT;
    mbar_wait(xbar, xpar);
    return false;
  }
  // [Z0, Z1] = C0^{-1} [g, t^{k+1}]
  {
    const float4* U[1] = {UP};
    float4* Yv[1] = {YP};
    df* Zv[2] = {Z0, Z1};
    c0inv_apply<1>(X, B, U, Yv, Zv);
  }
  // C0^{-1} (t^k - t^{k+1}) = z(t^k) - z(t^{k+1})
  if (b < B) Z2[b] = df_sub(ztk, Z1[b]);
  __syncthreads();
  __shared__ df s_W[9];
  __shared__ df s_A3[9];
  __shared__ df s_rhs[3];
  {
    // W = U^T C0^{-1} U is symmetric: its six distinct entries, one warp
    // each (one round for eight warps), mirrored below the diagonal
    const df* ua[6] = {U0, U0, U0, U1, U1, U2};
    const df* zb[6] = {Z0, Z1, Z2, Z1, Z2, Z2};
    __shared__ df s_w6[6];
    multi_dot_df(ua, zb, 6, B, s_w6);
    if (tid < 9) {
      const int i = tid / 3, j = tid % 3, a = min(i, j), c = max(i, j);
      s_W[tid] = s_w6[a == 0 ? c : (a == 1 ? 2 + c : 5)];
    }
    __syncthreads();
  }
  // C = C0 + U M U^T;  v = z_t - Z (I + M W)^{-1} M W[:, 1].  Warp 0: lane
  // (i, j) < 9 forms (I + M W)_ij, then the 3x3 system by Cramer's rule.
  if (tid < 32) {
    const int lane = tid;
    const df zero{0.f, 0.f};
    const df mb2 = df_mul(bbar, bbar);
    // M = [[0, -1, 0], [-1, var, 0], [0, 0, mean(beta)^2]]
    auto Mrow = [&](int i, int k) -> df {
      if (i == 0) return k == 1 ? df{-1.f, 0.f} : zero;
      if (i == 1) return k == 0 ? df{-1.f, 0.f} : (k == 1 ? var : zero);
      return k == 2 ? mb2 : zero;
    };
    if (lane < 9) {
      const int i = lane / 3, j = lane % 3;
      df a = (i == j) ? df{1.f, 0.f} : zero;
      for (int k = 0; k < 3; ++k) a = df_fma(Mrow(i, k), s_W[k * 3 + j], a);
      s_A3[lane] = a;
    } else if (lane < 12) {
      const int i = lane - 9;
      df r = zero;
      for (int k = 0; k < 3; ++k) r = df_fma(Mrow(i, k), s_W[k * 3 + 1], r);
      s_rhs[i] = r;
    }
    __syncwarp();
    // cofactors C_ij of A3 (lane i*3+j), determinant along row 0
    df cof = zero;
    if (lane < 9) {
      const int i = lane / 3, j = lane % 3;
      const int r0 = (i + 1) % 3, r1 = (i + 2) % 3, c0 = (j + 1) % 3, c1 = (j + 2) % 3;
      cof = df_sub(df_mul(s_A3[r0 * 3 + c0], s_A3[r1 * 3 + c1]),
                   df_mul(s_A3[r0 * 3 + c1], s_A3[r1 * 3 + c0]));
    }
    const df c00 = shfl_df(cof, 0), c01 = shfl_df(cof, 1), c02 = shfl_df(cof, 2);
    df det = df_mul(s_A3[0], c00);
    det = df_fma(s_A3[1], c01, det);
    det = df_fma(s_A3[2], c02, det);
    // y_i = sum_j C_ji rhs_j / det  (adjugate = transposed cofactors); all
    // lanes take part in the shuffles
    const df cf[9] = {shfl_df(cof, 0), shfl_df(cof, 1), shfl_df(cof, 2), shfl_df(cof, 3),
                      shfl_df(cof, 4), shfl_df(cof, 5), shfl_df(cof, 6), shfl_df(cof, 7),
                      shfl_df(cof, 8)};
    if (lane < 3) {
      const int i = lane;
      df num = df_mul(cf[0 * 3 + i], s_rhs[0]);
      num = df_fma(cf[1 * 3 + i], s_rhs[1], num);
      num = df_fma(cf[2 * 3 + i], s_rhs[2], num);
      s_y[i] = df_div(num, det);
    }
    if (lane == 0) {
      // Hadamard ratio |det| / prod ||row||: near 0 when I + M W is close to
      // singular, i.e. C^{k+1} is far more singular than C^0 along U; the
      // Woodbury form then loses the digits that a direct factorisation keeps
      float hr = 1.f;
      for (int i = 0; i < 3; ++i) {
        float n2 = 0.f;
        for (int j = 0; j < 3; ++j) n2 = fmaf(s_A3[i * 3 + j].hi, s_A3[i * 3 + j].hi, n2);
        hr *= sqrtf(n2);
      }
      hr = fabsf(det.hi) / fmaxf(hr, 1e-30f);
      s_bad = (!(det.hi > 0.f) || !df_isfinite(det)) ? 1 : (hr < 1e-8f ? 2 : 0);
      if (s_bad == 0 && p.force_direct) s_bad = 2;
      if (p.energy) {
        // objective at this iterate (Eq. (8) with the shrinkage step's
        // per-pixel form): sum_i (x_i - mu^k)^T (C^k)^-1 (x_i - mu^k)
        //   = N tr((C^k)^-1 S^k),  S^k = C^0 + (mu^0 - mu^k)(mu^0 - mu^k)^T,
        // mu^0 - mu^k = mean(beta) t^{k-1} = mean(beta) U e, e = (0, 1, 1);
        // with G = U^T (C^k)^-1 U = W (I + M W)^-1 (Woodbury) this is
        //   N (B - tr(G M) + mean(beta)^2 e^T G e)
        df G[9];
        const df idet = df_recip(det);
        for (int i = 0; i < 3; ++i)
          for (int j = 0; j < 3; ++j) {
            df g = zero;
            for (int k = 0; k < 3; ++k) g = df_fma(s_W[i * 3 + k], cf[j * 3 + k], g);
            G[i * 3 + j] = df_mul(g, idet);
          }
        df trGM = zero;
        for (int i = 0; i < 3; ++i)
          for (int j = 0; j < 3; ++j) trGM = df_fma(G[i * 3 + j], Mrow(j, i), trGM);
        const df eGe = df_add(df_add(G[4], G[5]), df_add(G[7], G[8]));
        const df per = df_add(df_sub(df{(float)B, 0.f}, trGM), df_mul(mb2, eGe));
        const double* dsn = p.dscal + (size_t)part * 4;
        double* en = p.energy + (size_t)part * p.energy_stride;
        en[pass] = s_bad == 0 ? dsn[DS_N] * df_to_double(per)
                              : __longlong_as_double(0x7ff8000000000000LL);
        en[pass - 1] += df_to_double(mom[B + 3]);  // the previous pass's pixel terms
      }
    }
  } else {
    // warps 1-7, idle while warp 0 solves: the outputs that do not depend
    // on its solution (the same on the direct path)
    for (int i = tid - 32; i < B; i += kThreads - 32) {
      stf(p.zt, pb + i, Z1[i]);
      stf(p.tprev, pb + i, U1[i]);
      stf(p.muk, pb + i, vmk[i]);
    }
  }
  __syncthreads();
  if (s_bad == 1) {
    fail_partition(p, part, false);
    return true;
  }
  if (s_bad == 2) {
    // direct path: C^{k+1} = C^0 + U M U^T assembled in double-float (into
    // the matrix region, no longer needed), factorised and solved
    const double* Sg = p.S + (size_t)part * B * B;
    const DfMat Xm{reinterpret_cast<float*>(X), B, B * B};
    const df mvar = var, mb2 = df_mul(bbar, bbar);
    for (int idx = tid; idx < B * B; idx += kThreads) {
      const int i = idx / B, j = idx % B;
      if (j < i) continue;  // upper triangle
      df c = df_from_double(Sg[idx]);
      c = df_sub(c, df_add(df_mul(U0[i], U1[j]), df_mul(U1[i], U0[j])));
      c = df_fma(mvar, df_mul(U1[i], U1[j]), c);
      c = df_fma(mb2, df_mul(U2[i], U2[j]), c);
      Xm.set(i, j, c);
    }
    if (!chol_inv_df(Xm, B, Y0)) {  // Y0 holds 1/diag(U)
      fail_partition(p, part, false);
      return true;
    }
    xtx_apply_df(Xm, B, Y0, U1, Y1, vv);
  } else {
    const df y0 = s_y[0], y1 = s_y[1], y2 = s_y[2];
    for (int i = tid; i < B; i += kThreads) {
      df zy = df_mul(Z0[i], y0);
      zy = df_fma(Z1[i], y1, zy);
      zy = df_fma(Z2[i], y2, zy);
      vv[i] = df_sub(Z1[i], zy);
    }
  }
  for (int i = tid; i < B; i += kThreads) U2[i] = df_sub(vmk[i], vmf[i]);  // mu^{k+1} - mu0f
  __syncthreads();
  __shared__ df s_d3[3];
  {
    const df* da[3] = {U1, vmf, U2};
    const df* db[3] = {vv, vv, vv};
    multi_dot_df(da, db, 3, B, s_d3);
  }
  const df q = s_d3[0], muv = s_d3[1], coff = s_d3[2];
  for (int i = tid; i < B; i += kThreads) p.vf[pb + i] = df_to_float(vv[i]);
  if (p.ck_vec && pass < p.ck_stages) {  // checkpoint of stage `pass`
    float2* cv = p.ck_vec + ((size_t)part * p.ck_stages + pass) * 4 * B;
    for (int i = tid; i < B; i += kThreads) {
      stf(cv, CKV_MU * B + i, vmk[i]);
      stf(cv, CKV_T * B + i, U1[i]);
      stf(cv, CKV_V * B + i, vv[i]);
      stf(cv, CKV_G * B + i, U0[i]);
    }
    if (tid == 0) {
      double* cs = p.ck_sc + ((size_t)part * p.ck_stages + pass) * 4;
      cs[CKS_Q] = df_to_double(q);
      cs[CKS_BBAR] = df_to_double(bbar);
      cs[CKS_VAR] = df_to_double(var);
    }
  }
  if (tid == 0) {
    float4* ps = reinterpret_cast<float4*>(p.pscal) + part;
    const float4 old = *ps;
    *ps = make_float4(df_to_float(q), df_to_float(muv), df_to_float(coff), old.w);
    double* dsw = p.dscal + (size_t)part * 4;
    dsw[DS_BBAR] = df_to_double(bbar);
    dsw[DS_Q] = df_to_double(q);
    if (!(q.hi > 0.f) || !df_isfinite(q)) p.status[part] = MF_ERR_NOT_SPD;
  }
  return true;
}

}  // namespace

}  // namespace mf
