// C ABI of the matched-filter library: plans, workspace and launch sequence.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/mf.h"
#include "mf_common.cuh"

namespace {

thread_local std::string g_last_error;

mf_status fail(mf_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return s;
}

#define MF_CUDA(call)                                                                  \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess)                                                             \
      return fail(MF_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_));        \
  } while (0)

int env_int(const char* name, int dflt) {
  const char* v = std::getenv(name);
  if (!v || !*v) return dflt;
  return std::atoi(v);
}

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

}  // namespace

namespace mf {
void set_last_error(const std::string& msg) { g_last_error = msg; }
}  // namespace mf

struct mf_plan_s {
  mf_desc d{};
  mf::Params prm{};       // geometry + workspace pointers; per-call fields set in retrieve
  void* ws = nullptr;
  size_t ws_bytes = 0;
  int nj = 0;             // template bucket
  size_t smem_stats = 0, smem_pixel = 0, smem_sinit = 0, smem_siter = 0, smem_slit = 0;
  int grid_stats = 0, grid_pixel = 0;
  // tensor maps of the last cube pointer (re-encoded when it changes)
  const float* map_cube = nullptr;
  CUtensorMap map_stats{}, map_pixel{};
  cudaStream_t last_stream = nullptr;
  int device = 0;
  int num_sms = 1;
  // host-I/O staging (mf_retrieve_host)
  float* h_cube = nullptr;
  uint8_t* h_mask = nullptr;
  float* h_k = nullptr;
  float* h_alpha = nullptr;
  // kernel timing (mf_profile)
  bool profile = false;
  struct Mark {
    int kind;
    cudaEvent_t start, stop;
  };
  std::vector<Mark> marks;
  size_t used = 0;
};

namespace {

int nj_bucket(int B4) {
  const int need = (B4 + 1) / 2;
  const int buckets[] = {1, 2, 4, 6, 8, 9, 10, 12, 16};
  for (int b : buckets)
    if (b >= need) return b;
  return -1;
}

// The shared-memory limit is an attribute of the kernel function, shared by
// every plan whose band count falls in the same template bucket (and every
// plan for the solve kernels): set it to the largest size any such plan needs.
cudaError_t set_attrs(const mf_plan_s* pl) {
  const int bmax_bucket = 8 * pl->nj;
  const int bmax = mf::kMaxB;
  const int ba = (bmax + 3 + 3) / 4 * 4;
  cudaError_t e = mf::stats_set_attributes(pl->nj, mf::stats_smem_bytes(bmax_bucket));
  if (e == cudaSuccess && pl->d.precision == MF_BF16SPLIT)
    e = mf::stats_tc_set_attributes(pl->nj, pl->smem_stats);
  if (e == cudaSuccess)
    e = mf::pixel_set_attributes(pl->nj, mf::pixel_smem_bytes(bmax_bucket, pl->nj));
  if (e == cudaSuccess)
    e = mf::solve_set_attributes(mf::solve_init_smem_bytes(bmax, ba), mf::solve_iter_smem_bytes(bmax),
                                 mf::solve_literal_smem_bytes(bmax, ba));
  return e;
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* ptr = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(ptr);
  }
  return fn;
}

// 3-D view (bands_total, cols, rows) of the cube with a box of
// (B, box_cols, box_rows) float32 elements; out-of-range boxes are zero filled
bool encode_cube_map(CUtensorMap* m, const mf::Params& p, const float* cube, int box_cols,
                     int box_rows) {
  auto fn = encode_fn();
  if (!fn) return false;
  const cuuint64_t dims[3] = {(cuuint64_t)p.bands_total, (cuuint64_t)p.cols, (cuuint64_t)p.rows};
  const cuuint64_t strides[2] = {(cuuint64_t)p.bands_total * sizeof(float),
                                 (cuuint64_t)p.bands_total * p.cols * sizeof(float)};
  const cuuint32_t box[3] = {(cuuint32_t)p.B, (cuuint32_t)box_cols, (cuuint32_t)box_rows};
  const cuuint32_t estr[3] = {1, 1, 1};
  const CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(cube), dims,
                        strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

constexpr size_t kMaxMarks = 1 << 14;

// events bracketing one launch when profiling; null when off or the pool is full
mf_plan_s::Mark* mark_begin(mf_plan_s* pl, int kind, cudaStream_t s) {
  if (!pl->profile) return nullptr;
  if (pl->used == pl->marks.size()) {
    if (pl->marks.size() >= kMaxMarks) return nullptr;
    mf_plan_s::Mark m{kind, nullptr, nullptr};
    if (cudaEventCreate(&m.start) != cudaSuccess) return nullptr;
    if (cudaEventCreate(&m.stop) != cudaSuccess) {
      cudaEventDestroy(m.start);
      return nullptr;
    }
    pl->marks.push_back(m);
  }
  mf_plan_s::Mark* m = &pl->marks[pl->used++];
  m->kind = kind;
  cudaEventRecord(m->start, s);
  return m;
}
void mark_end(mf_plan_s::Mark* m, cudaStream_t s) {
  if (m) cudaEventRecord(m->stop, s);
}

enum { KIND_STATS = 0, KIND_PIXEL = 1, KIND_SOLVE = 2, KIND_COUNT = 3 };

void stats_dispatch(mf_plan_s* pl, const mf::Params& prm, int mode, cudaStream_t s) {
  mf_plan_s::Mark* m = mark_begin(pl, KIND_STATS, s);
  if (pl->d.precision == MF_BF16SPLIT) {
    // persistent: one CTA per SM over the (column, chunk) work items
    if (mode == mf::STAT_INIT) mf::pilot_launch(s, prm);
    const int grid = std::min(pl->grid_stats, pl->num_sms);
    mf::stats_tc_launch(pl->nj, grid, pl->smem_stats, s, pl->map_stats, prm, mode);
  } else
    mf::stats_launch(pl->nj, pl->grid_stats, pl->smem_stats, s, pl->map_stats, prm, mode);
  mark_end(m, s);
}
void pixel_dispatch(mf_plan_s* pl, const mf::Params& prm, int mode, int acc, cudaStream_t s) {
  mf_plan_s::Mark* m = mark_begin(pl, KIND_PIXEL, s);
  mf::pixel_launch(pl->nj, pl->grid_pixel, pl->smem_pixel, s, pl->map_pixel, prm, mode, acc);
  mark_end(m, s);
}
void solve_init_dispatch(mf_plan_s* pl, const mf::Params& prm, cudaStream_t s) {
  mf_plan_s::Mark* m = mark_begin(pl, KIND_SOLVE, s);
  mf::solve_init_launch(pl->smem_sinit, s, prm);
  mark_end(m, s);
}
void solve_iter_dispatch(mf_plan_s* pl, const mf::Params& prm, int mode, cudaStream_t s) {
  mf_plan_s::Mark* m = mark_begin(pl, KIND_SOLVE, s);
  mf::solve_iter_launch(pl->smem_siter, s, prm, mode);
  mark_end(m, s);
}
void solve_literal_dispatch(mf_plan_s* pl, const mf::Params& prm, cudaStream_t s) {
  mf_plan_s::Mark* m = mark_begin(pl, KIND_SOLVE, s);
  mf::solve_literal_launch(pl->smem_slit, s, prm);
  mark_end(m, s);
}

}  // namespace

extern "C" {

const char* mf_status_string(mf_status s) {
  switch (s) {
    case MF_OK: return "ok";
    case MF_ERR_INVALID_ARG: return "invalid argument";
    case MF_ERR_CUDA: return "CUDA runtime error";
    case MF_ERR_OOM: return "out of device memory";
    case MF_ERR_NOT_SPD: return "covariance not positive definite (or N <= B)";
    case MF_ERR_NONFINITE_INPUT: return "non-finite scalar input";
    case MF_ERR_TIMEOUT: return "device-side wait timed out";
    case MF_ERR_INTERNAL: return "internal error";
    case MF_ERR_UNSUPPORTED: return "unsupported shape";
  }
  return "unknown status";
}

const char* mf_last_error(void) { return g_last_error.c_str(); }

mf_status mf_plan(const mf_desc* d, mf_plan_t* out) {
  g_last_error.clear();
  if (!d || !out) return fail(MF_ERR_INVALID_ARG, "null descriptor or output");
  *out = nullptr;
  if (d->rows <= 0 || d->cols <= 0 || d->bands_total <= 0)
    return fail(MF_ERR_INVALID_ARG, "rows, cols and bands_total must be positive");
  if (d->band_lo < 0 || d->band_hi > d->bands_total || d->band_hi <= d->band_lo)
    return fail(MF_ERR_INVALID_ARG, "band window [%d, %d) outside [0, %lld)", d->band_lo,
                d->band_hi, (long long)d->bands_total);
  if (d->col_group < 1) return fail(MF_ERR_INVALID_ARG, "col_group must be >= 1");
  if (d->layout != MF_BIP) return fail(MF_ERR_UNSUPPORTED, "only the BIP layout is supported");
  if (d->precision != MF_FP32 && d->precision != MF_BF16SPLIT)
    return fail(MF_ERR_INVALID_ARG, "unknown precision %d", d->precision);
  if (d->flags & ~(MF_ALBEDO | MF_SPARSE | MF_LITERAL | MF_PENALTY_NO_ALBEDO))
    return fail(MF_ERR_INVALID_ARG, "unknown flag bits 0x%x", d->flags);
  const int B = d->band_hi - d->band_lo;
  if (B < 8 || B > mf::kMaxB || B % 4 || d->band_lo % 4 || d->bands_total % 4)
    return fail(MF_ERR_UNSUPPORTED,
                "window of %d bands at %d in %lld: need 8 <= B <= %d and 16-byte aligned "
                "pixel windows (B, band_lo, bands_total multiples of 4)",
                B, d->band_lo, (long long)d->bands_total, mf::kMaxB);
  if (d->rows > (1LL << 30) || d->cols > (1LL << 24) || d->rows * d->cols > (1LL << 40))
    return fail(MF_ERR_UNSUPPORTED, "cube too large");
  if (d->precision == MF_BF16SPLIT && !mf::stats_tc_supported(B))
    return fail(MF_ERR_UNSUPPORTED, "MF_BF16SPLIT supports windows of 64 to 92 bands, got %d", B);

  mf_plan_s* pl = new mf_plan_s();
  pl->d = *d;
  mf::Params& p = pl->prm;
  p.rows = (int)d->rows;
  p.cols = (int)d->cols;
  p.bands_total = (int)d->bands_total;
  p.band_lo = d->band_lo;
  p.B = B;
  p.B4 = B / 4;
  p.G = (int)std::min<int64_t>(d->col_group, d->cols);
  p.P = (p.cols + p.G - 1) / p.G;
  p.BA = (B + 3 + 3) / 4 * 4;
  p.flags = d->flags;
  pl->nj = nj_bucket(p.B4);

  cudaError_t e = cudaGetDevice(&pl->device);
  if (e == cudaSuccess)
    e = cudaDeviceGetAttribute(&pl->num_sms, cudaDevAttrMultiProcessorCount, pl->device);
  if (e != cudaSuccess) {
    delete pl;
    return fail(MF_ERR_CUDA, "device query: %s", cudaGetErrorString(e));
  }
  // row blocking: pixel kernel blocks of rb rows (a multiple of the stage
  // height), as few as fill the SMs once (column tiles x row blocks ~ the
  // resident pixel CTAs per SM x SM count); statistics chunks sized so that the
  // statistics grid has several CTAs per SM
  p.n_ct = (p.cols + mf::kTileCols - 1) / mf::kTileCols;
  int rb = env_int("MF_RB_ROWS", 0);
  if (rb <= 0) {
    const long waves = (long)mf::pixel_ctas_per_sm(pl->nj) * pl->num_sms;
    const long nrb = std::max<long>(1, (waves + p.n_ct - 1) / p.n_ct);
    rb = (int)((p.rows + nrb - 1) / nrb);
  }
  rb = std::max(rb, mf::kStageRows);
  rb = (rb + mf::kStageRows - 1) / mf::kStageRows * mf::kStageRows;
  p.rb_rows = std::min(rb, (p.rows + mf::kStageRows - 1) / mf::kStageRows * mf::kStageRows);
  p.n_rb = (p.rows + p.rb_rows - 1) / p.rb_rows;
  int sc = env_int("MF_SC_ROWS", 0);
  if (sc <= 0) {
    const long target_ctas = 2400;
    long nsc = std::max<long>(1, (target_ctas + p.cols - 1) / p.cols);
    sc = (int)((p.rows + nsc - 1) / nsc);
    // the tensor-core form accumulates a chunk in float32 in tensor memory:
    // at most 1024 rows per chunk keeps that sum within the stated bound
    if (d->precision == MF_BF16SPLIT) sc = std::min(sc, 1024);
  }
  sc = std::max(mf::kStatRows, (sc + mf::kStatRows - 1) / mf::kStatRows * mf::kStatRows);
  p.sc_rows = sc;
  p.n_sc = (p.rows + p.sc_rows - 1) / p.sc_rows;
  pl->grid_stats = p.cols * p.n_sc;
  pl->grid_pixel = p.n_ct * p.n_rb;
  pl->smem_stats = d->precision == MF_BF16SPLIT ? mf::stats_tc_smem_bytes(B)
                                                 : mf::stats_smem_bytes(B);
  pl->smem_pixel = mf::pixel_smem_bytes(B, pl->nj);
  pl->smem_sinit = mf::solve_init_smem_bytes(B, p.BA);
  pl->smem_siter = mf::solve_iter_smem_bytes(B);
  pl->smem_slit = mf::solve_literal_smem_bytes(B, p.BA);

  // workspace
  const size_t P = (size_t)p.P;
  const size_t K1E = mf::k1_entries(p.BA), K3E = mf::k3_entries(B);
  struct Piece {
    void** dst;
    size_t bytes;
  };
  Piece pieces[] = {
      {(void**)&p.pilot, P * B * sizeof(float)},
      {(void**)&p.mu0, P * B * sizeof(float2)},
      {(void**)&p.mu0f, P * B * sizeof(float)},
      {(void**)&p.vf, P * B * sizeof(float)},
      {(void**)&p.zt, P * B * sizeof(float2)},
      {(void**)&p.tprev, P * B * sizeof(float2)},
      {(void**)&p.muk, P * B * sizeof(float2)},
      {(void**)&p.S, P * B * B * sizeof(double)},
      {(void**)&p.Linv, P * B * B * sizeof(float2)},
      {(void**)&p.pscal, P * 4 * sizeof(float)},
      {(void**)&p.dscal, P * 4 * sizeof(double)},
      {(void**)&p.k1part, P * p.G * p.n_sc * K1E * sizeof(float2)},
      {(void**)&p.k3part, P * p.G * p.n_rb * K3E * sizeof(float)},
      {(void**)&p.status, P * sizeof(int)},
  };
  size_t total = 0;
  for (auto& pc : pieces) total = align_up(total, 256) + align_up(pc.bytes, 256);
  e = cudaMalloc(&pl->ws, total);
  if (e != cudaSuccess) {
    delete pl;
    if (e == cudaErrorMemoryAllocation)
      return fail(MF_ERR_OOM, "workspace of %zu bytes: %s", total, cudaGetErrorString(e));
    return fail(MF_ERR_CUDA, "workspace allocation: %s", cudaGetErrorString(e));
  }
  pl->ws_bytes = total;
  size_t off = 0;
  for (auto& pc : pieces) {
    off = align_up(off, 256);
    *pc.dst = static_cast<char*>(pl->ws) + off;
    off += align_up(pc.bytes, 256);
  }
  e = cudaMemset(pl->ws, 0, total);
  if (e == cudaSuccess) e = set_attrs(pl);
  if (e != cudaSuccess) {
    cudaFree(pl->ws);
    delete pl;
    return fail(MF_ERR_CUDA, "plan set-up: %s", cudaGetErrorString(e));
  }
  *out = pl;
  return MF_OK;
}

void mf_destroy(mf_plan_t pl) {
  if (!pl) return;
  cudaDeviceSynchronize();
  for (auto& m : pl->marks) {
    cudaEventDestroy(m.start);
    cudaEventDestroy(m.stop);
  }
  cudaFree(pl->ws);
  cudaFree(pl->h_cube);
  cudaFree(pl->h_mask);
  cudaFree(pl->h_k);
  cudaFree(pl->h_alpha);
  delete pl;
}

int64_t mf_num_partitions(mf_plan_t pl) { return pl ? pl->prm.P : -1; }

mf_status mf_retrieve(mf_plan_t pl, const float* cube, const float* k, double lambda, double eps,
                      int32_t n_iter, const uint8_t* mask, const float* alpha_init,
                      float* alpha_out, float* albedo_out, void* stream) {
  g_last_error.clear();
  if (!pl) return fail(MF_ERR_INVALID_ARG, "null plan");
  if (!cube || !k || !alpha_out) return fail(MF_ERR_INVALID_ARG, "null cube, k or alpha_out");
  if (n_iter < 0 || n_iter > 100000) return fail(MF_ERR_INVALID_ARG, "n_iter = %d", n_iter);
  if (!std::isfinite(lambda) || !std::isfinite(eps))
    return fail(MF_ERR_NONFINITE_INPUT, "lambda or eps not finite");
  if (lambda < 0.0 || !(eps > 0.0))
    return fail(MF_ERR_INVALID_ARG, "need lambda >= 0 and eps > 0");
  if ((reinterpret_cast<uintptr_t>(cube) & 15) != 0)
    return fail(MF_ERR_INVALID_ARG, "cube must be 16-byte aligned");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  mf::Params p = pl->prm;
  p.cube = cube;
  p.k = k;
  p.mask = mask;
  p.alpha_init = alpha_init;
  p.alpha = alpha_out;
  p.albedo = albedo_out;
  p.lambda = (float)lambda;
  p.eps = (float)eps;
  p.n_iter = n_iter;
  const bool literal = (p.flags & MF_LITERAL) != 0;
  if (cube != pl->map_cube) {
    if (!encode_cube_map(&pl->map_stats, pl->prm, cube, 1, mf::kStatRows) ||
        !encode_cube_map(&pl->map_pixel, pl->prm, cube, mf::kTileCols, mf::kStageRows)) {
      pl->map_cube = nullptr;
      return fail(MF_ERR_CUDA, "cuTensorMapEncodeTiled failed for the cube");
    }
    pl->map_cube = cube;
  }
  MF_CUDA(cudaMemsetAsync(p.status, 0, (size_t)p.P * sizeof(int), s));
  stats_dispatch(pl, p, mf::STAT_INIT, s);
  solve_init_dispatch(pl, p, s);
  pixel_dispatch(pl, p, mf::PIX_INIT, n_iter > 0, s);
  for (int it = 1; it <= n_iter; ++it) {
    if (literal) {
      solve_iter_dispatch(pl, p, mf::SOLVE_MEAN_ONLY, s);
      stats_dispatch(pl, p, mf::STAT_LITERAL, s);
      solve_literal_dispatch(pl, p, s);
    } else {
      solve_iter_dispatch(pl, p, mf::SOLVE_FUSED, s);
    }
    pixel_dispatch(pl, p, mf::PIX_ITER, it < n_iter, s);
  }
  MF_CUDA(cudaGetLastError());
  pl->last_stream = s;
  return MF_OK;
}

mf_status mf_retrieve_host(mf_plan_t pl, const float* cube, const float* k, double lambda,
                           double eps, int32_t n_iter, const uint8_t* mask, float* alpha_out,
                           void* stream) {
  g_last_error.clear();
  if (!pl || !cube || !k || !alpha_out) return fail(MF_ERR_INVALID_ARG, "null argument");
  const mf::Params& g = pl->prm;
  const size_t npix = (size_t)g.rows * g.cols;
  const size_t cube_bytes = npix * g.bands_total * sizeof(float);
  if (!pl->h_cube) {
    MF_CUDA(cudaMalloc(&pl->h_cube, cube_bytes));
    MF_CUDA(cudaMalloc(&pl->h_mask, npix));
    MF_CUDA(cudaMalloc(&pl->h_k, (size_t)g.B * sizeof(float)));
    MF_CUDA(cudaMalloc(&pl->h_alpha, npix * sizeof(float)));
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  MF_CUDA(cudaMemcpyAsync(pl->h_cube, cube, cube_bytes, cudaMemcpyHostToDevice, s));
  MF_CUDA(cudaMemcpyAsync(pl->h_k, k, (size_t)g.B * sizeof(float), cudaMemcpyHostToDevice, s));
  if (mask) MF_CUDA(cudaMemcpyAsync(pl->h_mask, mask, npix, cudaMemcpyHostToDevice, s));
  mf_status st = mf_retrieve(pl, pl->h_cube, pl->h_k, lambda, eps, n_iter,
                             mask ? pl->h_mask : nullptr, nullptr, pl->h_alpha, nullptr, stream);
  if (st != MF_OK) return st;
  MF_CUDA(cudaMemcpyAsync(alpha_out, pl->h_alpha, npix * sizeof(float), cudaMemcpyDeviceToHost,
                          s));
  MF_CUDA(cudaStreamSynchronize(s));
  return MF_OK;
}

mf_status mf_background(mf_plan_t pl, double* mu0, double* cov0, void* stream) {
  g_last_error.clear();
  if (!pl || !mu0 || !cov0) return fail(MF_ERR_INVALID_ARG, "null argument");
  const mf::Params& p = pl->prm;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // mu0 is stored as double-float pairs: widen on the host side of the copy
  const size_t n = (size_t)p.P * p.B;
  std::vector<float2> tmp(n);
  MF_CUDA(cudaMemcpyAsync(tmp.data(), p.mu0, n * sizeof(float2), cudaMemcpyDeviceToHost, s));
  MF_CUDA(cudaStreamSynchronize(s));
  std::vector<double> mud(n);
  for (size_t i = 0; i < n; ++i) mud[i] = (double)tmp[i].x + (double)tmp[i].y;
  MF_CUDA(cudaMemcpyAsync(mu0, mud.data(), n * sizeof(double), cudaMemcpyHostToDevice, s));
  MF_CUDA(cudaStreamSynchronize(s));
  MF_CUDA(cudaMemcpyAsync(cov0, p.S, (size_t)p.P * p.B * p.B * sizeof(double),
                          cudaMemcpyDeviceToDevice, s));
  return MF_OK;
}

mf_status mf_profile(mf_plan_t pl, int32_t enable) {
  g_last_error.clear();
  if (!pl) return fail(MF_ERR_INVALID_ARG, "null plan");
  pl->profile = enable != 0;
  return MF_OK;
}

mf_status mf_profile_read(mf_plan_t pl, double* ms, int64_t* launches, int32_t n_kinds) {
  g_last_error.clear();
  if (!pl || !ms || !launches || n_kinds < 0) return fail(MF_ERR_INVALID_ARG, "bad argument");
  for (int i = 0; i < n_kinds; ++i) {
    ms[i] = 0.0;
    launches[i] = 0;
  }
  MF_CUDA(cudaStreamSynchronize(pl->last_stream));
  for (size_t i = 0; i < pl->used; ++i) {
    const auto& m = pl->marks[i];
    float t = 0.f;
    MF_CUDA(cudaEventElapsedTime(&t, m.start, m.stop));
    if (m.kind < n_kinds) {
      ms[m.kind] += t;
      launches[m.kind] += 1;
    }
  }
  pl->used = 0;
  return MF_OK;
}

mf_status mf_plan_status(mf_plan_t pl, int32_t* status) {
  g_last_error.clear();
  if (!pl || !status) return fail(MF_ERR_INVALID_ARG, "null argument");
  MF_CUDA(cudaStreamSynchronize(pl->last_stream));
  MF_CUDA(cudaMemcpy(status, pl->prm.status, (size_t)pl->prm.P * sizeof(int),
                     cudaMemcpyDeviceToHost));
  for (int i = 0; i < pl->prm.P; ++i)
    if (status[i] != MF_OK) return (mf_status)status[i];
  return MF_OK;
}

}  // extern "C"
