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
//          sum beta (rho - 1) and sum beta e_i (B-vector)
// with v = (C^k)^{-1} t(mu^k) and q = t^T v prepared by the previous tail.
//
// The last CTA of a partition then prepares the next pass:
//   mu^{k+1} = mu^0 - mean(beta) t^k                     (Eq. (10), exact)
//   C^{k+1}  = C^0 - (g t^T + t g^T) + mean(beta)^2 dd^T + var(beta) t t^T
//              with t = t^{k+1}, d = t^k - t^{k+1}, g = mean(beta (x - mu^0))
//   which is Eq. (11) expanded exactly: a rank-3 update U M U^T of C^0.
//   v = (C^{k+1})^{-1} t through C^0's Cholesky factor and the Woodbury
//   identity: v = z_t - Z (I + M Z^T U ...)^{-1} ..., all in float64.
// In the literal schedule the tail only forms mu^{k+1} and t^{k+1}; the
// statistics kernel then re-accumulates and refactorises C^{k+1}.
#include "mf_common.cuh"
#include "mf_pixel_io.cuh"
#include "../../include/mf.h"

namespace mf {

size_t pixel_smem_bytes(int B) { return (size_t)(12 * B + 64) * sizeof(double); }

__device__ void pixel_tail(const Params& p, int tail, int part, int ncp, double* sm,
                           double* red);

template <int NJ>
__global__ void __launch_bounds__(kThreads) pixel_kernel(Params p, int mode, int tail) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ __align__(16) float4 s_mu[kMaxB / 4];
  __shared__ __align__(16) float4 s_v[kMaxB / 4];
  __shared__ float s_red[kWarps][kMaxB + 4];
  __shared__ float s_sc[4];
  __shared__ int s_last, s_failed;
  __shared__ double s_dred[kWarps];

  int c, chunk;
  unit_of_block(p, p.n_rb, c, chunk);
  if (c >= p.cols) return;
  const int part = part_of(p, c);
  const int c0 = part * p.G;
  const int ncp = part_ncols(p, part);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int B = p.B, B4 = p.B4;
  const size_t pb = (size_t)part * B;

  for (int f = tid; f < B4; f += kThreads) {
    s_mu[f] = reinterpret_cast<const float4*>(p.mu0f + pb)[f];
    s_v[f] = reinterpret_cast<const float4*>(p.vf + pb)[f];
  }
  if (tid == 0) {
    const double* sc = p.scal + (size_t)part * SC_NSCAL;
    s_sc[0] = (float)sc[SC_Q];
    s_sc[1] = (float)sc[SC_MUV];
    s_sc[2] = (float)sc[SC_COFF];
    s_sc[3] = (float)sc[SC_INVMU2];
    s_failed = p.status[part] != MF_OK;
  }
  __syncthreads();
  const float q = s_sc[0], muv = s_sc[1], coff = s_sc[2], invmu2 = s_sc[3];
  const bool failed = s_failed != 0;
  const bool albedo = (p.flags & MF_ALBEDO) != 0;
  const bool sparse = (p.flags & MF_SPARSE) != 0;
  const bool pna = (p.flags & MF_PENALTY_NO_ALBEDO) != 0;
  const bool acc = tail != TAIL_NONE;
  const float lam = p.lambda, eps = p.eps;

  float g[NJ][4];
#pragma unroll
  for (int j = 0; j < NJ; ++j) g[j][0] = g[j][1] = g[j][2] = g[j][3] = 0.f;
  float sb = 0.f, sb2 = 0.f, sba = 0.f;

  const int r_beg = chunk * p.rb_rows;
  const int r_end = min(p.rows, r_beg + p.rb_rows);
  const int e = lane & 1;
  const int slot = lane >> 1;
  for (int r0 = r_beg + warp * 16; r0 < r_end; r0 += kWarps * 16) {
    const int row = r0 + slot;
    const bool inb = row < r_end;
    float4 x[NJ];
    const bool fin = load_pixel<NJ>(p, row, c, inb, e, x);
    const size_t pix = (size_t)(inb ? row : 0) * p.cols + c;
    const bool valid = inb && fin && (!p.mask || p.mask[pix] == 0);
    const float rho = pair_dot<NJ>(x, s_mu, e, B4) * invmu2;
    split_residual<NJ>(x, s_mu, rho, e, B4);
    const float pe = pair_dot<NJ>(x, s_v, e, B4);
    const float pp = pe + (rho - 1.f) * muv - coff;
    const float r = albedo ? rho : 1.f;
    float al;
    if (mode == PIX_INIT) {
      float a0;
      if (p.alpha_init)
        a0 = inb ? p.alpha_init[pix] : 0.f;
      else
        a0 = r > 0.f ? pp / (r * q) : 0.f;
      al = p.n_iter == 0 ? a0 : fmaxf(a0, 0.f);
    } else {
      const float ap = inb ? p.alpha[pix] : 0.f;
      const float w = sparse ? 1.f / (ap + eps) : 0.f;
      float pen = lam * w;
      if (pna) pen = r > 0.f ? pen / r : 0.f;
      al = r > 0.f ? fmaxf((pp - pen) / (r * q), 0.f) : 0.f;
    }
    if (!valid)
      al = 0.f;
    else if (failed)
      al = __int_as_float(0x7fc00000);
    if (inb && e == 0) {
      p.alpha[pix] = al;
      if (mode == PIX_INIT && p.albedo) p.albedo[pix] = valid ? r : 0.f;
    }
    if (acc) {
      const float beta = (valid && !failed && r > 0.f) ? r * al : 0.f;
      if (e == 0) {
        sb += beta;
        sb2 = fmaf(beta, beta, sb2);
        sba = fmaf(beta, rho - 1.f, sba);
      }
#pragma unroll
      for (int j = 0; j < NJ; ++j) {
        g[j][0] = fmaf(beta, x[j].x, g[j][0]);
        g[j][1] = fmaf(beta, x[j].y, g[j][1]);
        g[j][2] = fmaf(beta, x[j].z, g[j][2]);
        g[j][3] = fmaf(beta, x[j].w, g[j][3]);
      }
    }
  }
  if (!acc) return;

  // ---- CTA reduction of the moments (fixed order)
#pragma unroll
  for (int j = 0; j < NJ; ++j)
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      float v = g[j][u];
#pragma unroll
      for (int o = 2; o < 32; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      g[j][u] = v;
    }
  sb = warp_sumf(sb);
  sb2 = warp_sumf(sb2);
  sba = warp_sumf(sba);
  if (lane < 2) {
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
      const int f = lane + 2 * j;
      if (f < B4) {
#pragma unroll
        for (int u = 0; u < 4; ++u) s_red[warp][3 + 4 * f + u] = g[j][u];
      }
    }
    if (lane == 0) {
      s_red[warp][0] = sb;
      s_red[warp][1] = sb2;
      s_red[warp][2] = sba;
    }
  }
  __syncthreads();
  const int K3E = k3_entries(B);
  const int unit = (c - c0) * p.n_rb + chunk;
  float* dst = p.k3part + ((size_t)part * p.G * p.n_rb + unit) * K3E;
  for (int t = tid; t < B + 3; t += kThreads) {
    float s = 0.f;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) s += s_red[w][t];
    dst[t] = s;
  }
  __threadfence();
  __syncthreads();
  if (tid == 0) {
    const unsigned prev = atomicAdd(&p.counters[part], 1u);
    s_last = (prev + 1u == (unsigned)(ncp * p.n_rb)) ? 1 : 0;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  if (!failed) pixel_tail(p, tail, part, ncp, reinterpret_cast<double*>(smem_raw), s_dred);
  if (tid == 0) p.counters[part] = 0u;
}

// 3x3 solve with partial pivoting; returns det(A).
__device__ double solve3(double A[3][3], double b[3], double y[3]) {
  int perm[3] = {0, 1, 2};
  double det = 1.0;
  for (int col = 0; col < 3; ++col) {
    int piv = col;
    for (int r = col + 1; r < 3; ++r)
      if (fabs(A[r][col]) > fabs(A[piv][col])) piv = r;
    if (piv != col) {
      for (int k = 0; k < 3; ++k) {
        const double t = A[col][k];
        A[col][k] = A[piv][k];
        A[piv][k] = t;
      }
      const double t = b[col];
      b[col] = b[piv];
      b[piv] = t;
      const int tp = perm[col];
      perm[col] = perm[piv];
      perm[piv] = tp;
      det = -det;
    }
    det *= A[col][col];
    if (A[col][col] == 0.0) return 0.0;
    for (int r = col + 1; r < 3; ++r) {
      const double f = A[r][col] / A[col][col];
      for (int k = col; k < 3; ++k) A[r][k] -= f * A[col][k];
      b[r] -= f * b[col];
    }
  }
  for (int r = 2; r >= 0; --r) {
    double s = b[r];
    for (int k = r + 1; k < 3; ++k) s -= A[r][k] * y[k];
    y[r] = s / A[r][r];
  }
  return det;
}

__device__ void pixel_tail(const Params& p, int tail, int part, int ncp, double* sm,
                           double* red) {
  const int tid = threadIdx.x;
  const int B = p.B;
  const size_t pb = (size_t)part * B;
  const int K3E = k3_entries(B);
  double* mom = sm;               // B + 4 reduced moments
  double* U = mom + (B + 4);      // 3 x B: g, t^{k+1}, t^k - t^{k+1}
  double* Z = U + 3 * B;          // 3 x B: C0^{-1} U
  double* m0f = Z + 3 * B;        // mu0f
  double* mk = m0f + B;           // mu^{k+1}
  double* vv = mk + B;            // v
  double* dd = vv + B;            // mu^{k+1} - mu0f
  __shared__ double s_y[3];
  __shared__ int s_bad;

  const int nunits = ncp * p.n_rb;
  const float* P0 = p.k3part + (size_t)part * p.G * p.n_rb * K3E;
  for (int t = tid; t < B + 3; t += kThreads) {
    double s = 0.0;
    for (int u = 0; u < nunits; ++u) s += (double)__ldcg(P0 + (size_t)u * K3E + t);
    mom[t] = s;
  }
  __syncthreads();
  double* scal = p.scal + (size_t)part * SC_NSCAL;
  const double N = scal[SC_N];
  const double sb = mom[0], sb2 = mom[1], sba = mom[2];
  const double bbar = sb / N;
  const double var = sb2 / N - bbar * bbar;
  for (int b = tid; b < B; b += kThreads) {
    const double mu0 = p.mu0d[pb + b];
    const double mf = (double)p.mu0f[pb + b];
    const double tk = p.tprev[pb + b];
    const double muk1 = mu0 - bbar * tk;
    const double t1 = muk1 * (double)p.k[b];
    m0f[b] = mf;
    mk[b] = muk1;
    dd[b] = muk1 - mf;
    // g = mean(beta (x - mu0)), x - mu0 = e + (rho - 1) mu0f + (mu0f - mu0)
    U[b] = (mom[3 + b] + sba * mf + sb * (mf - mu0)) / N;
    U[B + b] = t1;
    U[2 * B + b] = tk - t1;
    Z[b] = U[b];
    Z[B + b] = t1;
    Z[2 * B + b] = tk - t1;
  }
  __syncthreads();
  if (tail == TAIL_LITERAL) {
    for (int b = tid; b < B; b += kThreads) {
      p.muk[pb + b] = mk[b];
      p.tprev[pb + b] = U[B + b];
    }
    if (tid == 0) scal[SC_BBAR] = bbar;
    return;
  }
  // Z = C0^{-1} U with C0 = L L^T (float64)
  block_chol_solve(p.L + pb * B, B, B, p.invd + pb, Z, B, 3);
  double W[3][3];
  for (int a = 0; a < 3; ++a)
    for (int b2 = 0; b2 < 3; ++b2) W[a][b2] = block_dot(U + a * B, Z + b2 * B, B, red);
  if (tid == 0) {
    // C = C0 + U M U^T; v = C^{-1} t = z_t - Z (I + M W)^{-1} M W[:,1]
    const double M[3][3] = {{0.0, -1.0, 0.0}, {-1.0, var, 0.0}, {0.0, 0.0, bbar * bbar}};
    double A3[3][3], rhs[3], y[3];
    for (int i = 0; i < 3; ++i) {
      rhs[i] = 0.0;
      for (int j = 0; j < 3; ++j) {
        double s = (i == j) ? 1.0 : 0.0;
        for (int k = 0; k < 3; ++k) s += M[i][k] * W[k][j];
        A3[i][j] = s;
        rhs[i] += M[i][j] * W[j][1];
      }
    }
    const double det = solve3(A3, rhs, y);
    s_bad = !(det > 0.0) || !isfinite(det);
    s_y[0] = y[0];
    s_y[1] = y[1];
    s_y[2] = y[2];
  }
  __syncthreads();
  if (s_bad) {
    if (tid == 0) p.status[part] = MF_ERR_NOT_SPD;
    return;
  }
  const double y0 = s_y[0], y1 = s_y[1], y2 = s_y[2];
  for (int b = tid; b < B; b += kThreads)
    vv[b] = Z[B + b] - (Z[b] * y0 + Z[B + b] * y1 + Z[2 * B + b] * y2);
  __syncthreads();
  const double qn = block_dot(U + B, vv, B, red);
  const double muv = block_dot(m0f, vv, B, red);
  const double coff = block_dot(dd, vv, B, red);
  for (int b = tid; b < B; b += kThreads) {
    p.vf[pb + b] = (float)vv[b];
    p.tprev[pb + b] = U[B + b];
    p.muk[pb + b] = mk[b];
  }
  if (tid == 0) {
    scal[SC_Q] = qn;
    scal[SC_MUV] = muv;
    scal[SC_COFF] = coff;
    scal[SC_BBAR] = bbar;
    if (!(qn > 0.0) || !isfinite(qn)) p.status[part] = MF_ERR_NOT_SPD;
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

void pixel_launch(int nj, int grid, size_t smem, cudaStream_t s, const Params& p, int mode,
                  int tail) {
#define MF_CASE(NJ)                                                   \
  case NJ:                                                            \
    pixel_kernel<NJ><<<grid, kThreads, smem, s>>>(p, mode, tail);     \
    return;
  switch (nj) { MF_NJ_CASES(MF_CASE) }
#undef MF_CASE
}

}  // namespace mf
