// Shared definitions of the matched-filter kernels (sm_103a).
//
// Data layout in HBM (one plan; P partitions, B bands in the window):
//   cube       caller's (rows, cols, bands_total) float32, BIP; window [band_lo, band_hi);
//              a batch of flightlines is stacked along rows (line l = rows
//              [row0_l, row0_l + rows_l)), each line with its own partitions
//   alpha      caller's (rows, cols) float32, updated in place every pass
//   lines      (n_lines) LineInfo      per-line geometry, lambda and iteration count
//   pilot      (P, K, B) float32     reference directions q_k of the statistics split
//   pilot_c    (P, K) float32        their offsets c_k (coefficients of the pilot mean)
//   pilot_s    (P, K) float32        their inverse squared norms 1 / (q_k . q_k)
//   mu0        (P, B) double-float   initial mean mu^0
//   mu0f       (P, B) float32        mu^0 rounded, as the pixel kernel holds it
//   vf         (P, B) float32        v = C^{-1} t of the current pass
//   zt         (P, B) double-float   C^0^{-1} t(mu^k) of the last statistics
//   tprev      (P, B) double-float   target t(mu^k) of the last statistics
//   muk        (P, B) double-float   mean mu^k (literal schedule)
//   S          (P, B, B) float64     C^0 (read back by mf_background)
//   Linv       (P, B, B + 1) double-float inverse of the Cholesky factor of C^0 (lower,
//              rows padded by one entry)
//   pscal      (P, 4) float32        q, mu0f.v, (mu^k - mu0f).v, 1/(mu0f.mu0f)
//   dscal      (P, 4) float64        N, mean(beta), q
//   k1part     (P, G * n_sc, K1E) double-float   per-CTA augmented second moments (the
//              tensor-core form stores a column-major BA x BA float Q in each unit)
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
// Reference directions of the statistics split: the float32 statistics use
// kDirsFp32 (an orthonormal basis of the partition's first valid pixels),
// the tensor-core form one (the mean of the first valid pixels)
constexpr int kDirsFp32 = 8;
constexpr int kMaxDirs = 8;
// augmented width of the moments: B bands, K direction coefficients, the
// target coefficient b and the constant 1, rounded up to a multiple of 4
__host__ __device__ inline int aug_width(int B, int K) { return (B + K + 2 + 3) / 4 * 4; }

enum : int { PS_Q = 0, PS_MUV, PS_COFF, PS_INVMU2, PS_N };
enum : int { DS_N = 0, DS_BBAR, DS_Q, DS_N2 };

enum : int { STAT_INIT = 0, STAT_LITERAL = 1 };
// Params::q_words: the 64-bit next-item counter, the abort word and a pad
// before the per-partition words
constexpr int kQueueHead = 4;
enum : int { PIX_INIT = 0, PIX_ITER = 1 };
enum : int { SOLVE_FUSED = 0, SOLVE_MEAN_ONLY = 1 };

// One flightline of a plan (a single retrieval has one).  Its statistics
// work items are (chunk, column), chunk-major, numbered from item0; its pixel
// CTAs are (row block, column tile), row-block-major, numbered from blk0; the
// per-CTA moment units of (column c, chunk) are k1u0 + c n_sc + chunk and of
// (column c, row block) k3u0 + c n_rb + rb, so a partition's units are
// contiguous.
struct LineInfo {
  int row0, rows;         // rows [row0, row0 + rows) of the stacked cube
  int n_sc, sc_rows;      // statistics chunks (sc_rows a multiple of kStatRows)
  int item0;              // first statistics item
  int n_rb, rb_rows;      // pixel row blocks (rb_rows a multiple of kStageRows)
  int blk0;               // first pixel CTA
  int n_iter;             // reweighting iterations N_iter of the line
  float lambda;           // multiplier on the weights of Eq. (5)
  int pad_;
  long long k1u0, k3u0;   // first moment units
};

struct Params {
  // geometry
  int rows, cols, bands_total, band_lo, B, B4, G;
  int Pl, P;              // partitions per line, in all lines
  int K;                  // reference directions of the statistics split (1..kMaxDirs)
  int BA;                 // augmented width: aug_width(B, K)
  int n_ct;               // pixel kernel column tiles
  int n_lines, n_items, n_blocks;  // lines; statistics items; pixel CTAs
  uint32_t flags;
  float eps;
  float l2_keep;          // backward pixel passes: fraction of each CTA's stages read
                          // last that are kept in L2 for the next pass (it walks the
                          // rows back)
  int force_direct;       // test hook (MF_FORCE_DIRECT=1 at plan creation): every fused
                          // iteration takes the direct factorisation of C^k
  long long test_wait;    // fault hook (MF_FAULT=timeout): > 0 makes every pixel CTA of
                          // pass 0 wait this many cycles on a barrier nothing arrives on
  int fault_notspd;       // fault hook (MF_FAULT=notspd): every initial factorisation fails
  int k1_colmajor;        // moment units hold Q (BA x BA floats, column-major, G = Q + Q^T;
                          // the tensor-core statistics) instead of the upper triangle of G in
                          // 4 x 4 blocks of double-float pairs (the float32 statistics)
  double* energy;         // optional: (P, energy_stride) objective per iterate (null = off)
  int energy_stride;      // n_iter + 1
  const LineInfo* lines;  // device, n_lines
  LineInfo line0;         // geometry of the only line of a single-line plan (its lambda and
                          // N_iter fields are not kept current: read those from `lines`)
  // caller buffers
  const float* cube;
  const float* k;
  const uint8_t* mask;
  const float* alpha_init;
  float* alpha;
  float* albedo;
  // workspace
  float* pilot;
  float* pilot_c;
  float* pilot_s;
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
  // checkpoints of a retrieval for the backward pass (null: none): alpha^k of
  // every pass k = 0..n, and per partition and pass the double-float vectors
  // mu^k, t^k, v^k, g^k and the scalars q^k, mean(beta)^k, var(beta)^k
  float* ck_alpha;      // (n + 1, rows, cols)
  float2* ck_vec;       // (P, n + 1, 4, B)
  double* ck_sc;        // (P, n + 1, 4)
  int ck_stages;        // n + 1
  // device timeline (mf_timeline; null: off): two words per launch, this
  // launch's at tl + 2 tl_slot
  unsigned long long* tl;
  int tl_slot;
  // launch with programmatic stream serialisation (see pdl_wait)
  int pdl;
  // the solve kernels prefetch into L2 the first pf_stages stages of every
  // pixel CTA of the pass that follows them (0: off; single-line plans)
  int pf_stages;
  // persistent work queue (MF_PERSISTENT, mf_queue.cu): q_words holds the
  // next item, the abort flag, per partition the passes whose solve has
  // completed (P) and per line and column tile the pixel items completed
  // over all passes (n_lines n_ct), zeroed before every retrieval; q_groups
  // the first item of each of the 2 n_lines groups of a pass, then the pass
  // size; q_wait_ns bounds each dependency wait
  int* q_words;
  const int* q_groups;
  long long q_wait_ns;
};

// Programmatic dependent launch.  A kernel launched with the programmatic
// stream-serialisation attribute may start while the kernel before it in
// the stream still runs: up to pdl_wait() it may only touch data no running
// kernel writes or reads (the cube, the mask, the plan's line table, and the
// outputs of kernels two or more launches back); pdl_wait() returns once
// the previous kernel has completed and its writes are visible.  Every
// kernel signals its dependents (pdl_trigger) only after its own wait, so at
// most two kernels overlap and everything two launches back is complete.
// Without the attribute both are no-ops.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// launch `kernel` on `s`, with the programmatic stream-serialisation
// attribute when `pdl` is set
template <typename... KArgs, typename... Args>
inline void launch_kernel(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                          cudaStream_t s, bool pdl, Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl ? 1 : 0;
  cudaLaunchKernelEx(&cfg, kernel, static_cast<Args&&>(args)...);
}

// Device timeline of a launch (mf_timeline).  When p.tl is set, thread 0 of
// every CTA folds %globaltimer (ns) at its start into slot[0] and at its exit
// into slot[1], both by atomicMax on zero-initialised words: slot[0] keeps
// the largest bitwise complement, i.e. the earliest start, slot[1] the
// latest exit, so the slot spans the launch from its first CTA's start to
// its last CTA's end.  One instance at the top of a kernel covers every
// return path.
__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
struct LaunchSpan {
  unsigned long long* s;
  __device__ explicit LaunchSpan(const Params& p, bool on = true)
      : s(on && p.tl && threadIdx.x == 0 ? p.tl + 2 * (size_t)p.tl_slot : nullptr) {
    if (s) atomicMax(s, ~globaltimer_ns());
  }
  __device__ ~LaunchSpan() {
    if (s) atomicMax(s + 1, globaltimer_ns());
  }
};

enum : int { CKV_MU = 0, CKV_T, CKV_V, CKV_G };
enum : int { CKS_Q = 0, CKS_BBAR, CKS_VAR };

// Backward pass of a single-line retrieval (see mf_backward.cu)
struct BwdParams {
  int n_iter;
  const float* grad_alpha;  // (rows, cols) adjoint of the output alpha^n
  float* abar[2];           // (rows, cols) partial adjoint of alpha^k, ping-pong by stage
  float* rbar;              // (rows, cols) adjoint of r_i, accumulated over stages
  float* coef;              // (n + 1, rows, cols, 2) cube-gradient coefficients, or null
  float* grad_cube;         // (rows, cols, B) output, or null
  float* vkf;               // (P, B) v^k of the current stage, float
  float* zf;                // (P, n + 1, B) zbar^k of every stage, float
  float* bpart;             // per-CTA partial sums of a backward pixel pass
  double* psc;              // (P, kPsc) per-partition scalars of the current stage
  float2* carry;            // (P, B) adjoint of t^{k-1} carried to stage k - 1
  float2* mubar0;           // (P, B) adjoint of mu^0
  double* sbar;             // (P, B) per-partition part of the gradient of s
  double* lbar;             // (P) per-partition part of the gradient of lambda
  float* mu0bar_n;          // (P, B) float: adjoint of mu^0 / N (cube gradient)
  float* grad_k;            // (B) output
  float* grad_lambda;       // (1) output
};
constexpr int kPsc = 16;
enum : int {
  PSC_Q = 0, PSC_MUV, PSC_COFF, PSC_INVM2, PSC_N, PSC_CNEXT, PSC_ZT, PSC_ZMU0, PSC_ZOFF,
  PSC_PSUM, PSC_QBAR, PSC_LAMBAR, PSC_BBAR
};
__host__ __device__ inline int bwd_entries(int B) { return B + 8; }

__host__ __device__ inline int k1_entries(int BA) {
  const int nb = BA / 4;
  return nb * (nb + 1) / 2 * 16;
}
// per pixel-kernel CTA and column: sum beta, sum beta^2, sum beta (rho - 1),
// sum beta e (B entries), and the pass's per-pixel energy terms (when asked)
__host__ __device__ inline int k3_entries(int B) { return B + 4; }

// partition of column c of line l; its line; its first column; its width
__device__ __forceinline__ int part_of(const Params& p, int l, int c) { return l * p.Pl + c / p.G; }
__device__ __forceinline__ int part_line(const Params& p, int part) { return part / p.Pl; }
__device__ __forceinline__ int part_col0(const Params& p, int part) { return (part % p.Pl) * p.G; }
__device__ __forceinline__ int part_ncols(const Params& p, int part) {
  return min(p.G, p.cols - part_col0(p, part));
}
// line of statistics item w / pixel CTA b (binary search over item0 / blk0)
__device__ __forceinline__ int line_of_item(const Params& p, int w) {
  int lo = 0, hi = p.n_lines - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (p.lines[mid].item0 <= w) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}
__device__ __forceinline__ int line_of_block(const Params& p, int b) {
  int lo = 0, hi = p.n_lines - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (p.lines[mid].blk0 <= b) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}
// statistics item w: line, column, chunk and its rows [r_beg, r_end)
struct StatItem {
  int line, c, chunk, r_beg, r_end;
  long long unit;  // moment unit
};
__device__ __forceinline__ StatItem stat_item(const Params& p, int w) {
  StatItem it;
  it.line = p.n_lines == 1 ? 0 : line_of_item(p, w);
  const LineInfo L = p.n_lines == 1 ? p.line0 : p.lines[it.line];
  const int local = w - L.item0;
  it.chunk = local / p.cols;
  it.c = local - it.chunk * p.cols;
  it.r_beg = L.row0 + it.chunk * L.sc_rows;
  it.r_end = min(L.row0 + L.rows, it.r_beg + L.sc_rows);
  it.unit = L.k1u0 + (long long)it.c * L.n_sc + it.chunk;
  return it;
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
size_t stats_smem_bytes(int B, int K);
size_t pixel_smem_bytes(int B, int nj);
int pixel_ctas_per_sm(int nj);  // resident pixel CTAs per SM for a template bucket
size_t solve_init_smem_bytes(int B, int BA);
size_t solve_iter_smem_bytes(int B);
size_t solve_literal_smem_bytes(int B, int BA);
cudaError_t stats_set_attributes(int nj, size_t smem);
cudaError_t pixel_set_attributes(int nj, size_t smem);
cudaError_t solve_set_attributes(size_t s_init, size_t s_iter, size_t s_lit);
// `pass`: 0 for the initial statistics / pixel pass, k for iteration k (lines
// with fewer iterations skip it)
void stats_launch(int nj, int grid, size_t smem, cudaStream_t s, const CUtensorMap& map,
                  const Params& p, int mode, int pass);
void pixel_launch(int nj, int grid, size_t smem, cudaStream_t s, const CUtensorMap& map,
                  const Params& p, int mode, int accumulate, int pass);
void solve_init_launch(size_t smem, cudaStream_t s, const Params& p);
void solve_iter_launch(size_t smem, cudaStream_t s, const Params& p, int mode, int pass);
void solve_literal_launch(size_t smem, cudaStream_t s, const Params& p, int pass);
size_t stats_tc_smem_bytes(int B);
bool stats_tc_supported(int B);
cudaError_t stats_tc_set_attributes(int nj, size_t smem);
void stats_tc_launch(int nj, int grid, size_t smem, cudaStream_t s, const CUtensorMap& map,
                     const Params& p, int mode, int pass);
void pilot_launch(cudaStream_t s, const Params& p);
void pilot_dirs_launch(cudaStream_t s, const Params& p);
void energy_final_launch(cudaStream_t s, const Params& p, int k);
// persistent work queue (mf_queue.cu)
cudaError_t queue_set_attributes(int nj, size_t smem);
int queue_ctas_per_sm(int nj, size_t smem);
void queue_launch(int nj, int grid, size_t smem, cudaStream_t s, const CUtensorMap& map,
                  const Params& p, int n_iter_max);
// backward pass (mf_backward.cu)
size_t bwd_pixel_smem_bytes(int B, int nj);
size_t bwd_solve_smem_bytes(int B);
cudaError_t bwd_set_attributes(int nj, size_t smem_pixel, size_t smem_solve);
void bwd_launch_stage(int nj, int grid_pixel, size_t smem_pixel, size_t smem_solve,
                      cudaStream_t s, const CUtensorMap& map, const Params& p,
                      const BwdParams& b, int stage);
void bwd_launch_final(int nj, size_t smem_pixel, cudaStream_t s, const Params& p,
                      const BwdParams& b);
size_t background_smem_bytes(int B, int BA);
cudaError_t background_set_attributes(size_t smem);
void background_launch(size_t smem, cudaStream_t s, const Params& p, double* mu, double* cov);
}  // namespace mf

#include <string>
namespace mf {
// message returned by mf_last_error() on the calling thread (defined in mf_api.cu)
void set_last_error(const std::string& msg);

}  // namespace mf
