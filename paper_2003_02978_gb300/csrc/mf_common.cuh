// Shared definitions of the matched-filter kernels (sm_103a).
//
// Data layout in HBM (one plan):
//   cube      caller's (rows, cols, bands_total) float32, BIP; window [band_lo, band_hi)
//   alpha     caller's (rows, cols) float32, updated in place every pass
//   mu0d/mu0f (P, B) float64 / float32  initial mean mu^0 of each partition
//   vf        (P, B) float32            C^{-1} t of the current pass, for the pixel kernel
//   tprev     (P, B) float64            target t(mu^k) of the last statistics
//   muk       (P, B) float64            mean mu^k (literal schedule)
//   S, L      (P, B, B) float64         C^0 and the Cholesky factor in use (lower)
//   invd      (P, B) float64            1 / diag(L)
//   scal      (P, NSCAL) float64        per-partition scalars (q, offsets, N, ...)
//   k1part    (P, G * n_sc, K1P) float64  per-CTA augmented second moments
//   k3part    (P, G * n_rb, K3P) float32  per-CTA enhancement moments
//   counters  (P) uint32                arrival counters (last CTA runs the tail)
//   status    (P) int32                 mf_status per partition
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace mf {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kColGroup = 8;        // adjacent columns swept together (coalesced alpha/mask)
constexpr int kMaxB = 128;

// per-partition scalars
enum : int {
  SC_Q = 0,      // q = t^T C^-1 t (the normaliser of the shrinkage step)
  SC_MUV,        // mu0f . v
  SC_COFF,       // (mu^k - mu0f) . v
  SC_N,          // valid pixel count N
  SC_INVMU2,     // 1 / (mu0f . mu0f)
  SC_BBAR,       // mean(beta) of the last update
  SC_NSCAL = 8
};

enum : int { STAT_INIT = 0, STAT_LITERAL = 1 };        // statistics kernel modes
enum : int { PIX_INIT = 0, PIX_ITER = 1 };             // pixel kernel modes
enum : int { TAIL_NONE = 0, TAIL_FUSED = 1, TAIL_LITERAL = 2 };

struct Params {
  // geometry
  int rows, cols, bands_total, band_lo, B, B4, G, P;
  int rb_rows, n_rb;      // pixel kernel row blocks
  int sc_rows, n_sc;      // statistics kernel row chunks
  int BA;                 // augmented width: roundup4(B + 3)
  uint32_t flags;
  int n_iter;
  float lambda, eps;      // as the kernels use them (float32)
  // caller buffers
  const float* cube;
  const float* k;
  const uint8_t* mask;
  const float* alpha_init;
  float* alpha;
  float* albedo;
  // workspace
  double* mu0d;
  float* mu0f;
  float* vf;
  double* tprev;
  double* muk;
  double* S;
  double* L;
  double* invd;
  double* scal;
  double* k1part;
  float* k3part;
  unsigned* counters;
  int* status;
};

__host__ __device__ inline int k1_entries(int BA) {
  const int nb = BA / 4;
  return nb * (nb + 1) / 2 * 16;
}
__host__ __device__ inline int k3_entries(int B) { return B + 4; }

__device__ __forceinline__ int part_of(const Params& p, int c) { return c / p.G; }
__device__ __forceinline__ int part_ncols(const Params& p, int part) {
  const int c0 = part * p.G;
  return min(p.G, p.cols - c0);
}

// Grid decomposition shared by both streaming kernels: CTAs walk groups of
// kColGroup adjacent columns; inside a group, all row chunks of the group,
// columns fastest.  Neighbouring columns of the same rows run together (their
// alpha / mask sectors are shared in L2) and partitions complete in order.
__device__ __forceinline__ void unit_of_block(const Params& p, int nchunks, int& c, int& chunk) {
  const int idx = blockIdx.x;
  const int ci = idx % kColGroup;
  const int rest = idx / kColGroup;
  chunk = rest % nchunks;
  const int cg = rest / nchunks;
  c = cg * kColGroup + ci;
}

__device__ __forceinline__ const float* pixel_ptr(const Params& p, int row, int col) {
  return p.cube + ((size_t)row * p.cols + col) * p.bands_total + p.band_lo;
}

__device__ __forceinline__ bool finite4(float4 v) {
  return isfinite(v.x) && isfinite(v.y) && isfinite(v.z) && isfinite(v.w);
}

// ----------------------------------------------------------- block helpers
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_sumf(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum over the whole CTA; every thread gets the result.  `red` holds kWarps doubles.
__device__ inline double block_sum(double v, double* red) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < kWarps; ++i) s += red[i];
  return s;
}

// Dot product of two length-n vectors in shared memory (fixed order per thread).
__device__ inline double block_dot(const double* a, const double* b, int n, double* red) {
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += kThreads) s += a[i] * b[i];
  return block_sum(s, red);
}

// In-place Cholesky A = L L^T of the leading n x n block (row stride ld) in
// shared memory, right-looking, one column per step.  Writes 1/L_jj to invd.
// Returns false (uniformly across the CTA) if a pivot is not > 0 or not finite.
__device__ inline bool block_cholesky(double* A, int n, int ld, double* invd, int* flag) {
  const int tid = threadIdx.x;
  if (tid == 0) *flag = 0;
  for (int j = 0; j < n; ++j) {
    __syncthreads();
    if (tid == 0) {
      double d = A[j * ld + j];
      if (!(d > 0.0) || !isfinite(d)) {
        *flag = 1;
        d = 1.0;
      }
      const double s = sqrt(d);
      A[j * ld + j] = s;
      invd[j] = 1.0 / s;
    }
    __syncthreads();
    if (*flag) return false;
    const double id = invd[j];
    for (int i = j + 1 + tid; i < n; i += kThreads) A[i * ld + j] *= id;
    __syncthreads();
    const int m = n - j - 1;
    const int cnt = m * (m + 1) / 2;
    for (int idx = tid; idx < cnt; idx += kThreads) {
      int ii = (int)((sqrtf(8.0f * (float)idx + 1.0f) - 1.0f) * 0.5f);
      while (ii * (ii + 1) / 2 > idx) --ii;
      while ((ii + 1) * (ii + 2) / 2 <= idx) ++ii;
      const int kk = idx - ii * (ii + 1) / 2;
      const int i = j + 1 + ii, k = j + 1 + kk;
      A[i * ld + k] -= A[i * ld + j] * A[k * ld + j];
    }
  }
  __syncthreads();
  return true;
}

// Solve (L L^T) X = X in place for nrhs right-hand sides stored as rows of X
// (X[r * ldx + i]).  L lower, row stride ld, 1/diag in invd.  L may live in
// shared or global memory.
__device__ inline void block_chol_solve(const double* L, int n, int ld, const double* invd,
                                        double* X, int ldx, int nrhs) {
  const int tid = threadIdx.x;
  // forward: L y = b
  for (int j = 0; j < n; ++j) {
    __syncthreads();
    if (tid < nrhs) X[tid * ldx + j] *= invd[j];
    __syncthreads();
    const int m = n - j - 1;
    for (int idx = tid; idx < m * nrhs; idx += kThreads) {
      const int r = idx / m, i = j + 1 + idx % m;
      X[r * ldx + i] -= L[i * ld + j] * X[r * ldx + j];
    }
  }
  // backward: L^T z = y
  for (int j = n - 1; j >= 0; --j) {
    __syncthreads();
    if (tid < nrhs) X[tid * ldx + j] *= invd[j];
    __syncthreads();
    for (int idx = tid; idx < j * nrhs; idx += kThreads) {
      const int r = idx / j, i = idx % j;
      X[r * ldx + i] -= L[j * ld + i] * X[r * ldx + j];
    }
  }
  __syncthreads();
}

// ------------------------------------------------------- host-side launchers
// (each defined in the translation unit that defines the kernel)
size_t stats_smem_bytes(int B, int BA);
size_t pixel_smem_bytes(int B);
cudaError_t stats_set_attributes(int nj, size_t smem);
cudaError_t pixel_set_attributes(int nj, size_t smem);
void stats_launch(int nj, int grid, size_t smem, cudaStream_t s, const Params& p, int mode);
void pixel_launch(int nj, int grid, size_t smem, cudaStream_t s, const Params& p, int mode,
                  int tail);

}  // namespace mf
