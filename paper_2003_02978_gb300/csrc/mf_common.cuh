// Shared definitions of the matched-filter kernels (sm_103a).
//
// Data layout in HBM (one plan; P partitions, B bands in the window):
//   cube       caller's (rows, cols, bands_total) float32, BIP; window [band_lo, band_hi)
//   alpha      caller's (rows, cols) float32, updated in place every pass
//   pilot      (P, B) float32        reference direction m of the initial statistics
//   mu0        (P, B) double-float   initial mean mu^0
//   mu0f       (P, B) float32        mu^0 rounded, as the pixel kernel holds it
//   vf         (P, B) float32        v = C^{-1} t of the current pass
//   zt         (P, B) double-float   C^0^{-1} t(mu^k) of the last statistics
//   tprev      (P, B) double-float   target t(mu^k) of the last statistics
//   muk        (P, B) double-float   mean mu^k (literal schedule)
//   S          (P, B, B) float64     C^0 (read back by mf_background)
//   Linv       (P, B, B) double-float inverse of the Cholesky factor of C^0 (lower)
//   pscal      (P, 4) float32        q, mu0f.v, (mu^k - mu0f).v, 1/(mu0f.mu0f)
//   dscal      (P, 4) float64        N, mean(beta), q
//   k1part     (P, G * n_sc, K1E) double-float   per-CTA augmented second moments
//   k3part     (P, G * n_rb, K3E) float32        per-CTA enhancement moments
//   status     (P) int32             mf_status per partition
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace mf {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kMaxB = 128;
constexpr int kTileCols = 16;     // pixel kernel: adjacent columns per tile (one lane pair each)
constexpr int kStageRows = 8;     // pixel kernel: rows per pipeline stage (one per consumer warp)
constexpr int kStatRows = 128;    // statistics kernel: rows per pipeline stage

enum : int { PS_Q = 0, PS_MUV, PS_COFF, PS_INVMU2, PS_N };
enum : int { DS_N = 0, DS_BBAR, DS_Q, DS_N2 };

enum : int { STAT_INIT = 0, STAT_LITERAL = 1 };
enum : int { PIX_INIT = 0, PIX_ITER = 1 };
enum : int { SOLVE_FUSED = 0, SOLVE_MEAN_ONLY = 1 };

struct Params {
  // geometry
  int rows, cols, bands_total, band_lo, B, B4, G, P;
  int rb_rows, n_rb;      // pixel kernel row blocks (multiple of kStageRows)
  int sc_rows, n_sc;      // statistics kernel row chunks (multiple of kStatRows)
  int BA;                 // augmented width: roundup4(B + 3)
  int n_ct;               // pixel kernel column tiles
  uint32_t flags;
  int n_iter;
  float lambda, eps;
  // caller buffers
  const float* cube;
  const float* k;
  const uint8_t* mask;
  const float* alpha_init;
  float* alpha;
  float* albedo;
  // workspace
  float* pilot;
  float2* mu0;
  float* mu0f;
  float* vf;
  float2* zt;
  float2* tprev;
  float2* muk;
  double* S;
  float2* Linv;
  float* pscal;
  double* dscal;
  float2* k1part;
  float* k3part;
  int* status;
};

__host__ __device__ inline int k1_entries(int BA) {
  const int nb = BA / 4;
  return nb * (nb + 1) / 2 * 16;
}
__host__ __device__ inline int k3_entries(int B) { return B + 4; }

__device__ __forceinline__ int part_of(const Params& p, int c) { return c / p.G; }
__device__ __forceinline__ int part_ncols(const Params& p, int part) {
  return min(p.G, p.cols - part * p.G);
}

__device__ __forceinline__ const float* pixel_ptr(const Params& p, int row, int col) {
  return p.cube + ((size_t)row * p.cols + col) * p.bands_total + p.band_lo;
}

__device__ __forceinline__ bool finite4(float4 v) {
  return isfinite(v.x) && isfinite(v.y) && isfinite(v.z) && isfinite(v.w);
}

__device__ __forceinline__ float warp_sumf(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// thread t < nb(nb+1)/2 owns the 4x4 block (bi, bj), bi <= bj, of the
// augmented second-moment matrix
__host__ __device__ inline void block_of(int t, int nb, int& bi, int& bj) {
  int r = 0, rem = t;
  while (rem >= nb - r) {
    rem -= nb - r;
    ++r;
  }
  bi = r;
  bj = r + rem;
}

// ------------------------------------------------------- host-side launchers
// (each defined in the translation unit that defines the kernel)
size_t stats_smem_bytes(int B);
size_t pixel_smem_bytes(int B, int nj);
int pixel_ctas_per_sm(int nj);  // resident pixel CTAs per SM for a template bucket
size_t solve_init_smem_bytes(int B, int BA);
size_t solve_iter_smem_bytes(int B);
size_t solve_literal_smem_bytes(int B, int BA);
cudaError_t stats_set_attributes(int nj, size_t smem);
cudaError_t pixel_set_attributes(int nj, size_t smem);
cudaError_t solve_set_attributes(size_t s_init, size_t s_iter, size_t s_lit);
void stats_launch(int nj, int grid, size_t smem, cudaStream_t s, const CUtensorMap& map,
                  const Params& p, int mode);
void pixel_launch(int nj, int grid, size_t smem, cudaStream_t s, const CUtensorMap& map,
                  const Params& p, int mode, int accumulate);
void solve_init_launch(size_t smem, cudaStream_t s, const Params& p);
void solve_iter_launch(size_t smem, cudaStream_t s, const Params& p, int mode);
void solve_literal_launch(size_t smem, cudaStream_t s, const Params& p);
size_t stats_tc_smem_bytes(int B);
bool stats_tc_supported(int B);
cudaError_t stats_tc_set_attributes(int nj, size_t smem);
void stats_tc_launch(int nj, int grid, size_t smem, cudaStream_t s, const CUtensorMap& map,
                     const Params& p, int mode);
void pilot_launch(cudaStream_t s, const Params& p);
size_t background_smem_bytes(int B, int BA);
cudaError_t background_set_attributes(size_t smem);
void background_launch(size_t smem, cudaStream_t s, const Params& p, double* mu, double* cov);
}  // namespace mf

#include <string>
namespace mf {
// message returned by mf_last_error() on the calling thread (defined in mf_api.cu)
void set_last_error(const std::string& msg);

}  // namespace mf
