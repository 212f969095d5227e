// Statistics kernel: background mean and covariance of each partition.
//
// Fig. 1 (Algorithm AlbedoReWeightL1Filter) initialises mu^0 = (1/N) sum L_i
// and C^0 = (1/N) sum (L_i - mu^0)(L_i - mu^0)^T (outer product, as in
// Eq. (11)); the literal schedule recomputes C^k = (1/N) sum d_i d_i^T with
// d_i = L_i - r_i alpha_i^{k-1} t(mu^k) - mu^k at every iteration.
//
// One pass over the cube.  Each pixel is split along a reference direction m
// (the first valid pixel of the partition at initialisation, mu^0 afterwards):
//   x_i = rho_i m + e_i,  rho_i = x_i.m / m.m,
// which removes the large albedo component (Sec. II-C) from what is
// accumulated in float32: the CTA forms the augmented second moments of
//   [e_i, a_i, b_i, 1],  a_i = rho_i - 1,  b_i = -r_i alpha_i^{k-1},
// (a symmetric (B+3)x(B+3) product, 4x4 register blocks per thread), folds
// each 128-pixel batch into float-float (TwoSum) accumulators and writes
// them as float64.  The last CTA of a partition reduces all partial moments
// in a fixed order in float64, assembles C exactly from them, factorises it
// (Cholesky, float64) and solves C v = t.
#include "mf_common.cuh"
#include "mf_pixel_io.cuh"
#include "../../include/mf.h"

namespace mf {

constexpr int kBatch = 128;

size_t stats_smem_bytes(int B, int BA) {
  const size_t stage = (size_t)kBatch * BA * sizeof(float);
  const size_t tail = ((size_t)BA * BA + 8 * (size_t)B + 16) * sizeof(double);
  return stage > tail ? stage : tail;
}

// thread t < nb(nb+1)/2 owns the 4x4 block (bi, bj), bi <= bj
__device__ __forceinline__ void block_of(int t, int nb, int& bi, int& bj) {
  int r = 0, rem = t;
  while (rem >= nb - r) {
    rem -= nb - r;
    ++r;
  }
  bi = r;
  bj = r + rem;
}

__device__ __forceinline__ void two_sum_acc(float& hi, float& lo, float x) {
  const float s = hi + x;
  const float bp = s - hi;
  const float err = (hi - (s - bp)) + (x - bp);
  hi = s;
  lo += err;
}

__device__ void stats_tail(const Params& p, int mode, int part, int ncp, const float* s_ref,
                           double* sm, double* red, int* flag);

template <int NJ>
__global__ void __launch_bounds__(kThreads) stats_kernel(Params p, int mode) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* stage = reinterpret_cast<float*>(smem_raw);
  __shared__ __align__(16) float s_ref[kMaxB];
  __shared__ float s_inv_ref2;
  __shared__ int s_last, s_flag, s_pilot;
  __shared__ double s_red[kWarps];

  int c, chunk;
  unit_of_block(p, p.n_sc, c, chunk);
  if (c >= p.cols) return;
  const int part = part_of(p, c);
  const int c0 = part * p.G;
  const int ncp = part_ncols(p, part);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int B = p.B, B4 = p.B4, BA = p.BA;

  // ---- reference direction m
  if (mode == STAT_INIT) {
    if (warp == 0) {
      // first valid pixel of the partition in row-major order
      long found = -1;
      const long total = (long)p.rows * ncp;
      for (long base = 0; base < total && found < 0; base += 32) {
        const long i = base + lane;
        bool ok = false;
        if (i < total) {
          const int row = (int)(i / ncp), col = c0 + (int)(i % ncp);
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
      if (pi >= 0) {
        const int row = pi / ncp, col = c0 + pi % ncp;
        v = pixel_ptr(p, row, col)[b];
      }
      s_ref[b] = v;
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
      s_inv_ref2 = (float)p.scal[(size_t)part * SC_NSCAL + SC_INVMU2];
    }
  }
  __syncthreads();
  const float inv_ref2 = s_inv_ref2;
  const float4* ref4 = reinterpret_cast<const float4*>(s_ref);
  const bool albedo = (p.flags & MF_ALBEDO) != 0;

  // ---- SYRK ownership
  const int nb = BA / 4;
  const int nblk = nb * (nb + 1) / 2;
  int bi = 0, bj = 0;
  const bool syrk = tid < nblk;
  if (syrk) block_of(tid, nb, bi, bj);
  float hi[16], lo[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) hi[i] = lo[i] = 0.f;

  const int r_beg = chunk * p.sc_rows;
  const int r_end = min(p.rows, r_beg + p.sc_rows);
  const int e = lane & 1;
  const int slot = warp * 16 + (lane >> 1);
  for (int r0 = r_beg; r0 < r_end; r0 += kBatch) {
    // stage the augmented vectors [e_i, a_i, b_i, 1] of 128 pixels
    {
      const int row = r0 + slot;
      const bool inb = row < r_end;
      float4 x[NJ];
      const bool fin = load_pixel<NJ>(p, row, c, inb, e, x);
      const size_t pix = (size_t)(inb ? row : 0) * p.cols + c;
      const bool valid = inb && fin && (!p.mask || p.mask[pix] == 0);
      const float rho = pair_dot<NJ>(x, ref4, e, B4) * inv_ref2;
      split_residual<NJ>(x, ref4, rho, e, B4);
      float bcoef = 0.f;
      if (mode == STAT_LITERAL && valid) {
        const float r = albedo ? rho : 1.f;
        bcoef = r > 0.f ? -(r * p.alpha[pix]) : 0.f;
      }
      float* dst = stage + (size_t)slot * BA;
#pragma unroll
      for (int j = 0; j < NJ; ++j) {
        const int f = e + 2 * j;
        if (f < B4) {
          float4 v = valid ? x[j] : make_float4(0.f, 0.f, 0.f, 0.f);
          *reinterpret_cast<float4*>(dst + 4 * f) = v;
        }
      }
      if (e == 0) {
        dst[B] = valid ? rho - 1.f : 0.f;
        dst[B + 1] = valid ? bcoef : 0.f;
        dst[B + 2] = valid ? 1.f : 0.f;
        for (int q = B + 3; q < BA; ++q) dst[q] = 0.f;
      }
    }
    __syncthreads();
    if (syrk) {
      float acc[16];
#pragma unroll
      for (int i = 0; i < 16; ++i) acc[i] = 0.f;
      const float* col_i = stage + 4 * bi;
      const float* col_j = stage + 4 * bj;
#pragma unroll 4
      for (int s = 0; s < kBatch; ++s) {
        const float4 va = *reinterpret_cast<const float4*>(col_i + (size_t)s * BA);
        const float4 vb = *reinterpret_cast<const float4*>(col_j + (size_t)s * BA);
        const float a4[4] = {va.x, va.y, va.z, va.w};
        const float b4[4] = {vb.x, vb.y, vb.z, vb.w};
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int w = 0; w < 4; ++w) acc[u * 4 + w] = fmaf(a4[u], b4[w], acc[u * 4 + w]);
      }
#pragma unroll
      for (int i = 0; i < 16; ++i) two_sum_acc(hi[i], lo[i], acc[i]);
    }
    __syncthreads();
  }

  // ---- publish this CTA's moments
  const int K1E = k1_entries(BA);
  const int unit = (c - c0) * p.n_sc + chunk;
  double* dst = p.k1part + ((size_t)part * p.G * p.n_sc + unit) * K1E;
  if (syrk) {
#pragma unroll
    for (int i = 0; i < 16; ++i) dst[tid * 16 + i] = (double)hi[i] + (double)lo[i];
  }
  __threadfence();
  __syncthreads();
  if (tid == 0) {
    const unsigned prev = atomicAdd(&p.counters[part], 1u);
    s_last = (prev + 1u == (unsigned)(ncp * p.n_sc)) ? 1 : 0;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  stats_tail(p, mode, part, ncp, s_ref, reinterpret_cast<double*>(smem_raw), s_red, &s_flag);
  if (tid == 0) p.counters[part] = 0u;
}

// Reduce the partition's partial moments, assemble C, factorise, solve C v = t.
__device__ void stats_tail(const Params& p, int mode, int part, int ncp, const float* s_ref,
                           double* sm, double* red, int* flag) {
  const int tid = threadIdx.x;
  const int B = p.B, BA = p.BA;
  const int K1E = k1_entries(BA);
  const int nb = BA / 4;
  double* A = sm;                    // BA x BA
  double* u1 = A + (size_t)BA * BA;  // reference direction
  double* u2 = u1 + B;               // target t^k (literal) / 0
  double* u3 = u2 + B;               // u1 - mu
  double* mu = u3 + B;               // mean of the statistics
  double* vz = mu + B;               // right-hand side / solution
  double* id = vz + B;               // 1 / diag(L)
  double* tt = id + B;               // target of the solve

  const int nunits = ncp * p.n_sc;
  const double* P0 = p.k1part + (size_t)part * p.G * p.n_sc * K1E;
  for (int q = tid; q < K1E; q += kThreads) {
    double s = 0.0;
    for (int u = 0; u < nunits; ++u) s += __ldcg(P0 + (size_t)u * K1E + q);
    const int t = q >> 4, w = q & 15;
    int bi, bj;
    block_of(t, nb, bi, bj);
    const int i = 4 * bi + (w >> 2), j = 4 * bj + (w & 3);
    A[i * BA + j] = s;
    A[j * BA + i] = s;
  }
  __syncthreads();
  const double N = A[(B + 2) * BA + (B + 2)];
  const bool enough = N > (double)B;
  const double iN = enough ? 1.0 / N : 0.0;
  const size_t pb = (size_t)part * B;
  for (int b = tid; b < B; b += kThreads) {
    if (mode == STAT_INIT) {
      const double m = (double)s_ref[b];
      u1[b] = m;
      u2[b] = 0.0;
      mu[b] = m + (A[b * BA + B + 2] + A[B * BA + B + 2] * m) * iN;
      u3[b] = m - mu[b];
    } else {
      u1[b] = (double)p.mu0f[pb + b];
      u2[b] = p.tprev[pb + b];
      mu[b] = p.muk[pb + b];
      u3[b] = u1[b] - mu[b];
    }
  }
  __syncthreads();
  // C = (1/N) sum (e + a u1 + b u2 + u3)(...)^T, expanded over the moments
  const double aa = A[B * BA + B], ab = A[B * BA + B + 1], bb = A[(B + 1) * BA + B + 1];
  const double a1 = A[B * BA + B + 2], b1 = A[(B + 1) * BA + B + 2];
  const double n1 = A[(B + 2) * BA + B + 2];
  for (int idx = tid; idx < B * B; idx += kThreads) {
    const int i = idx / B, j = idx % B;
    double v = A[i * BA + j];
    v += A[i * BA + B] * u1[j] + u1[i] * A[j * BA + B];
    v += A[i * BA + B + 1] * u2[j] + u2[i] * A[j * BA + B + 1];
    v += A[i * BA + B + 2] * u3[j] + u3[i] * A[j * BA + B + 2];
    v += aa * u1[i] * u1[j] + ab * (u1[i] * u2[j] + u2[i] * u1[j]) + bb * u2[i] * u2[j];
    v += a1 * (u1[i] * u3[j] + u3[i] * u1[j]) + b1 * (u2[i] * u3[j] + u3[i] * u2[j]);
    v += n1 * u3[i] * u3[j];
    A[i * BA + j] = v * iN;
  }
  __syncthreads();
  double* Sg = p.S + (size_t)part * B * B;
  if (mode == STAT_INIT) {
    for (int idx = tid; idx < B * B; idx += kThreads) Sg[idx] = A[(idx / B) * BA + idx % B];
  }
  const bool ok = enough && block_cholesky(A, B, BA, id, flag);
  double* scal = p.scal + (size_t)part * SC_NSCAL;
  if (!ok) {
    for (int b = tid; b < B; b += kThreads) {
      p.vf[pb + b] = 0.f;
      if (mode == STAT_INIT) {
        p.mu0f[pb + b] = 0.f;
        p.mu0d[pb + b] = 0.0;
        p.tprev[pb + b] = 0.0;
      }
    }
    if (tid == 0) {
      p.status[part] = MF_ERR_NOT_SPD;
      scal[SC_Q] = 1.0;
      scal[SC_MUV] = 0.0;
      scal[SC_COFF] = 0.0;
      if (mode == STAT_INIT) {
        scal[SC_N] = N;
        scal[SC_INVMU2] = 0.0;
      }
    }
    return;
  }
  double* Lg = p.L + (size_t)part * B * B;
  for (int idx = tid; idx < B * B; idx += kThreads) {
    const int i = idx / B, j = idx % B;
    Lg[idx] = (j <= i) ? A[i * BA + j] : 0.0;
  }
  for (int b = tid; b < B; b += kThreads) {
    p.invd[pb + b] = id[b];
    const double t = (mode == STAT_INIT) ? mu[b] * (double)p.k[b] : u2[b];
    tt[b] = t;
    vz[b] = t;
  }
  block_chol_solve(A, B, BA, id, vz, B, 1);
  // mu0f as the pixel kernel will hold it
  for (int b = tid; b < B; b += kThreads) {
    if (mode == STAT_INIT) {
      const float mf = (float)mu[b];
      p.mu0f[pb + b] = mf;
      p.mu0d[pb + b] = mu[b];
      p.tprev[pb + b] = tt[b];
      u1[b] = (double)mf;           // now mu0f
    }
    u3[b] = mu[b] - u1[b];          // mu^k - mu0f
  }
  __syncthreads();
  const double q = block_dot(tt, vz, B, red);
  const double muv = block_dot(u1, vz, B, red);
  const double coff = block_dot(u3, vz, B, red);
  const double n2 = block_dot(u1, u1, B, red);
  for (int b = tid; b < B; b += kThreads) p.vf[pb + b] = (float)vz[b];
  if (tid == 0) {
    scal[SC_Q] = q;
    scal[SC_MUV] = muv;
    scal[SC_COFF] = coff;
    if (mode == STAT_INIT) {
      scal[SC_N] = N;
      scal[SC_INVMU2] = n2 > 0.0 ? 1.0 / n2 : 0.0;
      scal[SC_BBAR] = 0.0;
      p.status[part] = (q > 0.0 && isfinite(q)) ? MF_OK : MF_ERR_NOT_SPD;
    } else if (!(q > 0.0 && isfinite(q))) {
      p.status[part] = MF_ERR_NOT_SPD;
    }
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

void stats_launch(int nj, int grid, size_t smem, cudaStream_t s, const Params& p, int mode) {
#define MF_CASE(NJ)                                                   \
  case NJ:                                                            \
    stats_kernel<NJ><<<grid, kThreads, smem, s>>>(p, mode);           \
    return;
  switch (nj) { MF_NJ_CASES(MF_CASE) }
#undef MF_CASE
}

}  // namespace mf
