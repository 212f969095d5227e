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
  // persistent work queue (MF_PERSISTENT): one launch after the statistics
  bool persistent = false;
  size_t smem_queue = 0, q_bytes = 0;
  int grid_queue = 0;
  // flightlines: host copy of the device table, pinned staging for the
  // per-call lambda / iteration counts, and the values last uploaded
  int n_lines = 1;
  std::vector<mf::LineInfo> lines;
  mf::LineInfo* lines_pinned = nullptr;
  cudaEvent_t lines_copied = nullptr;
  bool lines_valid = false;
  // CUDA graph of the whole retrieval (re-captured when a pointer, the pass
  // count or eps changes); captured on a plan-owned stream, launched on the
  // caller's
  struct GraphKey {
    const void* ptr[6];
    int n_iter;
    float eps;
    bool timeline;
    bool operator==(const GraphKey& o) const {
      for (int i = 0; i < 6; ++i)
        if (ptr[i] != o.ptr[i]) return false;
      return n_iter == o.n_iter && eps == o.eps && timeline == o.timeline;
    }
  };
  // the last checkpointed forward (mf_retrieve_train), for mf_retrieve_backward
  struct Train {
    const void* ckpt = nullptr;
    int n_iter = 0;
    bool cube_grad = false;
    const float* cube = nullptr;
    const float* k = nullptr;
    const uint8_t* mask = nullptr;
    double eps = 0.0;
  } train;
  bool use_graph = true;
  // launch every kernel but a retrieval's first with programmatic stream
  // serialisation (MF_PDL=0 at plan creation: off)
  bool pdl = true;
  cudaStream_t cap_stream = nullptr;
  // two graphs (keyed by pointers, pass count, eps, timeline): the
  // double-buffered host entry point alternates between two sets of buffers
  static constexpr int kGraphs = 2;
  cudaGraphExec_t gexec[kGraphs] = {};
  GraphKey gkey[kGraphs]{};
  int gnext = 0;  // the slot a new key replaces
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
  // double-buffered staging of mf_retrieve_host_async: slot b's device
  // buffers, a copy stream, and per slot the events "copied in" and
  // "consumed" (its retrieval and the copy of alpha out have finished)
  float* a_cube[2] = {nullptr, nullptr};
  uint8_t* a_mask[2] = {nullptr, nullptr};
  float* a_k[2] = {nullptr, nullptr};
  float* a_alpha[2] = {nullptr, nullptr};
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t copied[2] = {nullptr, nullptr}, consumed[2] = {nullptr, nullptr};
  int aslot = 0;
  // kernel timing (mf_profile)
  bool profile = false;
  struct Mark {
    int kind;
    cudaEvent_t start, stop;
  };
  std::vector<Mark> marks;
  size_t used = 0;
  // device timeline (mf_timeline): one slot of two words per launch of the
  // last enqueued retrieval (graph replays reuse the captured slots), and the
  // kind of each slot's launch
  bool timeline = false;
  unsigned long long* tl_dev = nullptr;
  std::vector<int> tl_kind;
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
  const int ba = mf::aug_width(bmax, mf::kMaxDirs);
  cudaError_t e = mf::stats_set_attributes(pl->nj, mf::stats_smem_bytes(bmax_bucket, mf::kDirsFp32));
  if (e == cudaSuccess && pl->d.precision == MF_BF16SPLIT)
    e = mf::stats_tc_set_attributes(pl->nj, pl->smem_stats);
  if (e == cudaSuccess)
    e = mf::pixel_set_attributes(pl->nj, mf::pixel_smem_bytes(bmax_bucket, pl->nj));
  if (e == cudaSuccess)
    e = mf::solve_set_attributes(mf::solve_init_smem_bytes(bmax, ba), mf::solve_iter_smem_bytes(bmax),
                                 mf::solve_literal_smem_bytes(bmax, ba));
  if (e == cudaSuccess && pl->persistent)
    e = mf::queue_set_attributes(
        pl->nj, std::max({mf::pixel_smem_bytes(bmax_bucket, pl->nj), mf::solve_init_smem_bytes(bmax, ba),
                          mf::solve_iter_smem_bytes(bmax)}));
  return e;
}

// resolved once (a function-local static's initialisation is thread safe)
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static const PFN_cuTensorMapEncodeTiled_v12000 fn = []() {
    void* ptr = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(ptr);
    return (PFN_cuTensorMapEncodeTiled_v12000) nullptr;
  }();
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

enum { KIND_STATS = 0, KIND_PIXEL = 1, KIND_SOLVE = 2, KIND_QUEUE = 3, KIND_COUNT = 4 };

constexpr size_t kMaxSpans = 4096;  // device timeline slots (launches per retrieval)

// a launch's Params: with the device timeline on, its own slot; `first`:
// the retrieval's first kernel, which follows a memset, not a kernel, and is
// launched without the programmatic attribute
mf::Params span_params(mf_plan_s* pl, const mf::Params& prm, int kind, bool first = false) {
  mf::Params q = prm;
  q.pdl = pl->pdl && !first;
  q.tl = nullptr;
  if (pl->timeline && pl->tl_dev && pl->tl_kind.size() < kMaxSpans) {
    q.tl = pl->tl_dev;
    q.tl_slot = (int)pl->tl_kind.size();
    pl->tl_kind.push_back(kind);
  }
  return q;
}

void stats_dispatch(mf_plan_s* pl, const mf::Params& prm, int mode, int pass, cudaStream_t s) {
  mf_plan_s::Mark* m = mark_begin(pl, KIND_STATS, s);
  if (pl->d.precision == MF_BF16SPLIT) {
    // persistent: one CTA per SM over the (column, chunk) work items
    if (mode == mf::STAT_INIT) mf::pilot_launch(s, span_params(pl, prm, KIND_STATS, true));
    const int grid = std::min(pl->grid_stats, pl->num_sms);
    mf::stats_tc_launch(pl->nj, grid, pl->smem_stats, s, pl->map_stats,
                        span_params(pl, prm, KIND_STATS), mode, pass);
  } else {
    if (mode == mf::STAT_INIT) mf::pilot_dirs_launch(s, span_params(pl, prm, KIND_STATS, true));
    mf::stats_launch(pl->nj, pl->grid_stats, pl->smem_stats, s, pl->map_stats,
                     span_params(pl, prm, KIND_STATS), mode, pass);
  }
  mark_end(m, s);
}
void pixel_dispatch(mf_plan_s* pl, const mf::Params& prm, int mode, int acc, int pass,
                    cudaStream_t s) {
  mf_plan_s::Mark* m = mark_begin(pl, KIND_PIXEL, s);
  mf::pixel_launch(pl->nj, pl->grid_pixel, pl->smem_pixel, s, pl->map_pixel,
                   span_params(pl, prm, KIND_PIXEL), mode, acc, pass);
  mark_end(m, s);
}
void solve_init_dispatch(mf_plan_s* pl, const mf::Params& prm, cudaStream_t s) {
  mf_plan_s::Mark* m = mark_begin(pl, KIND_SOLVE, s);
  mf::solve_init_launch(pl->smem_sinit, s, span_params(pl, prm, KIND_SOLVE));
  mark_end(m, s);
}
void solve_iter_dispatch(mf_plan_s* pl, const mf::Params& prm, int mode, int pass,
                         cudaStream_t s) {
  mf_plan_s::Mark* m = mark_begin(pl, KIND_SOLVE, s);
  mf::solve_iter_launch(pl->smem_siter, s, span_params(pl, prm, KIND_SOLVE), mode, pass);
  mark_end(m, s);
}
void queue_dispatch(mf_plan_s* pl, const mf::Params& prm, int n_iter_max, cudaStream_t s) {
  mf_plan_s::Mark* m = mark_begin(pl, KIND_QUEUE, s);
  mf::queue_launch(pl->nj, pl->grid_queue, pl->smem_queue, s, pl->map_pixel,
                   span_params(pl, prm, KIND_QUEUE, true), n_iter_max);
  mark_end(m, s);
}
void solve_literal_dispatch(mf_plan_s* pl, const mf::Params& prm, int pass, cudaStream_t s) {
  mf_plan_s::Mark* m = mark_begin(pl, KIND_SOLVE, s);
  mf::solve_literal_launch(pl->smem_slit, s, span_params(pl, prm, KIND_SOLVE), pass);
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

}  // extern "C"

namespace {

// Validate the descriptor and build a plan over n_lines flightlines stacked
// along rows (line_rows[l] rows each; d->rows is their sum).
mf_status build_plan(const mf_desc* d, const int64_t* line_rows, int n_lines,
                     const mf_tuning* tune, mf_plan_t* out) {
  if (!d || !out) return fail(MF_ERR_INVALID_ARG, "null descriptor or output");
  *out = nullptr;
  if (d->rows <= 0 || d->cols <= 0 || d->bands_total <= 0)
    return fail(MF_ERR_INVALID_ARG, "rows, cols and bands_total must be positive");
  if (n_lines < 1 || n_lines > (1 << 20)) return fail(MF_ERR_INVALID_ARG, "n_lines = %d", n_lines);
  int64_t sum = 0;
  for (int l = 0; l < n_lines; ++l) {
    if (line_rows[l] <= 0) return fail(MF_ERR_INVALID_ARG, "line %d has %lld rows", l,
                                       (long long)line_rows[l]);
    sum += line_rows[l];
  }
  if (sum != d->rows)
    return fail(MF_ERR_INVALID_ARG, "rows %lld != sum of the line rows %lld", (long long)d->rows,
                (long long)sum);
  if (d->band_lo < 0 || d->band_hi > d->bands_total || d->band_hi <= d->band_lo)
    return fail(MF_ERR_INVALID_ARG, "band window [%d, %d) outside [0, %lld)", d->band_lo,
                d->band_hi, (long long)d->bands_total);
  if (d->col_group < 1) return fail(MF_ERR_INVALID_ARG, "col_group must be >= 1");
  if (d->layout != MF_BIP) return fail(MF_ERR_UNSUPPORTED, "only the BIP layout is supported");
  if (d->precision != MF_FP32 && d->precision != MF_BF16SPLIT)
    return fail(MF_ERR_INVALID_ARG, "unknown precision %d", d->precision);
  if (d->flags & ~(MF_ALBEDO | MF_SPARSE | MF_LITERAL | MF_PENALTY_NO_ALBEDO | MF_PERSISTENT))
    return fail(MF_ERR_INVALID_ARG, "unknown flag bits 0x%x", d->flags);
  if ((d->flags & MF_PERSISTENT) && (d->flags & MF_LITERAL))
    return fail(MF_ERR_INVALID_ARG, "MF_PERSISTENT runs the fused schedule, not MF_LITERAL");
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

  // fault hook: MF_FAULT=alloc fails here as an exhausted device would,
  // before any CUDA call; =notspd and =timeout are set in the plan below
  const char* fault = std::getenv("MF_FAULT");
  const std::string fault_s = fault ? fault : "";
  if (fault_s == "alloc")
    return fail(MF_ERR_OOM, "workspace allocation refused (fault hook MF_FAULT=alloc)");
  if (!fault_s.empty() && fault_s != "notspd" && fault_s != "timeout")
    return fail(MF_ERR_INVALID_ARG, "MF_FAULT=%s: expected alloc, notspd or timeout",
                fault_s.c_str());

  mf_plan_s* pl = new mf_plan_s();
  pl->d = *d;
  pl->n_lines = n_lines;
  mf::Params& p = pl->prm;
  p.rows = (int)d->rows;
  p.cols = (int)d->cols;
  p.bands_total = (int)d->bands_total;
  p.band_lo = d->band_lo;
  p.B = B;
  p.B4 = B / 4;
  p.G = (int)std::min<int64_t>(d->col_group, d->cols);
  p.Pl = (p.cols + p.G - 1) / p.G;
  p.P = n_lines * p.Pl;
  // reference directions of the statistics split: one for the tensor-core
  // form, kDirsFp32 for the float32 statistics
  p.K = d->precision == MF_BF16SPLIT ? 1 : mf::kDirsFp32;
  p.BA = mf::aug_width(B, p.K);
  p.k1_colmajor = d->precision == MF_BF16SPLIT;
  p.flags = d->flags;
  p.n_lines = n_lines;
  pl->nj = nj_bucket(p.B4);
  pl->persistent = (d->flags & MF_PERSISTENT) != 0;
  pl->use_graph = env_int("MF_GRAPH", 1) != 0;
  pl->pdl = env_int("MF_PDL", 1) != 0;
  p.pf_stages = env_int("MF_PF_STAGES", 4);
  if (tune && tune->use_graph < 0) pl->use_graph = false;

  cudaError_t e = cudaGetDevice(&pl->device);
  if (e == cudaSuccess)
    e = cudaDeviceGetAttribute(&pl->num_sms, cudaDevAttrMultiProcessorCount, pl->device);
  if (e != cudaSuccess) {
    delete pl;
    return fail(MF_ERR_CUDA, "device query: %s", cudaGetErrorString(e));
  }
  // Row blocking.  Pixel kernel: blocks of about h_p rows (a multiple of the
  // stage height), as few as fill the SMs once (column tiles x row blocks ~
  // the resident pixel CTAs per SM x SM count), at most 512 rows so that a
  // batch of long lines has no long CTAs at its end.  Statistics: chunks of
  // about h_s rows so that the SIMT grid has several CTAs per SM, at most
  // 1024 rows in the tensor-core form (float32 sums in tensor memory) and
  // 2048 otherwise.  Every line is split evenly into whole blocks / chunks.
  p.n_ct = (p.cols + mf::kTileCols - 1) / mf::kTileCols;
  // test hook: every fused iteration through the direct factorisation
  p.force_direct = env_int("MF_FORCE_DIRECT", 0) != 0;
  // fault hooks: every initial factorisation reported not positive definite;
  // every pixel CTA of pass 0 runs out of a 2000-cycle wait
  p.fault_notspd = fault_s == "notspd";
  p.test_wait = fault_s == "timeout" ? 2000 : 0;
  {
    // the share of the cube that a backward pixel pass leaves in L2 for the
    // next one: about 3/4 of the L2 (the rest holds the pass's writes and
    // moments)
    int dev = 0, l2 = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev);
    const double cube = (double)p.rows * p.cols * (d->band_hi - d->band_lo) * sizeof(float);
    p.l2_keep = cube > 0 ? (float)std::min(1.0, 0.75 * l2 / cube) : 0.f;
  }
  int hp = tune && tune->pixel_rows > 0 ? tune->pixel_rows : env_int("MF_RB_ROWS", 0);
  if (hp <= 0) {
    const long waves = (long)mf::pixel_ctas_per_sm(pl->nj) * pl->num_sms;
    const long nrb = std::max<long>(1, (waves + p.n_ct - 1) / p.n_ct);
    hp = (int)std::min<long>(512, (p.rows + nrb - 1) / nrb);
  }
  hp = std::max(hp, mf::kStageRows);
  int hs = tune && tune->stat_rows > 0 ? tune->stat_rows : env_int("MF_SC_ROWS", 0);
  if (hs <= 0) {
    // the float32 statistics kernel runs one CTA per item and wants many;
    // the tensor-core one is persistent (one CTA per SM walking the items),
    // balanced with about eight items per SM, and longer items (up to 1024
    // rows) mean fewer per-item epilogues and moment partials
    const bool tc = d->precision == MF_BF16SPLIT;
    const long target_items = tc ? 8L * pl->num_sms : 2400;
    const long nsc = std::max<long>(1, (target_items + p.cols - 1) / p.cols);
    hs = (int)std::min<long>(tc ? 1024 : 2048, (p.rows + nsc - 1) / nsc);
  }
  hs = std::max(hs, mf::kStatRows);
  auto round_up = [](int x, int m) { return (x + m - 1) / m * m; };
  pl->lines.resize(n_lines);
  int row0 = 0;
  long long items = 0, blocks = 0, k1u = 0, k3u = 0;
  for (int l = 0; l < n_lines; ++l) {
    mf::LineInfo& L = pl->lines[l];
    L = mf::LineInfo{};
    L.row0 = row0;
    L.rows = (int)line_rows[l];
    L.n_sc = (L.rows + hs - 1) / hs;
    L.sc_rows = round_up((L.rows + L.n_sc - 1) / L.n_sc, mf::kStatRows);
    L.n_sc = (L.rows + L.sc_rows - 1) / L.sc_rows;
    L.n_rb = (L.rows + hp - 1) / hp;
    L.rb_rows = round_up((L.rows + L.n_rb - 1) / L.n_rb, mf::kStageRows);
    L.n_rb = (L.rows + L.rb_rows - 1) / L.rb_rows;
    L.item0 = (int)items;
    L.blk0 = (int)blocks;
    L.k1u0 = k1u;
    L.k3u0 = k3u;
    L.n_iter = 0;
    L.lambda = 0.f;
    items += (long long)p.cols * L.n_sc;
    blocks += (long long)p.n_ct * L.n_rb;
    k1u += (long long)p.cols * L.n_sc;
    k3u += (long long)p.cols * L.n_rb;
    row0 += L.rows;
  }
  if (items > INT32_MAX || blocks > INT32_MAX) {
    delete pl;
    return fail(MF_ERR_UNSUPPORTED, "batch too large for one launch grid");
  }
  p.n_items = (int)items;
  p.n_blocks = (int)blocks;
  p.line0 = pl->lines[0];
  pl->grid_stats = p.n_items;
  pl->grid_pixel = p.n_blocks;
  pl->smem_stats = d->precision == MF_BF16SPLIT ? mf::stats_tc_smem_bytes(B)
                                                 : mf::stats_smem_bytes(B, p.K);
  pl->smem_pixel = mf::pixel_smem_bytes(B, pl->nj);
  pl->smem_sinit = mf::solve_init_smem_bytes(B, p.BA);
  pl->smem_siter = mf::solve_iter_smem_bytes(B);
  pl->smem_slit = mf::solve_literal_smem_bytes(B, p.BA);

  // workspace
  const size_t P = (size_t)p.P;
  const size_t K1E = mf::k1_entries(p.BA), K3E = mf::k3_entries(B);
  mf::LineInfo* lines_d = nullptr;
  struct Piece {
    void** dst;
    size_t bytes;
  };
  Piece pieces[] = {
      {(void**)&lines_d, (size_t)n_lines * sizeof(mf::LineInfo)},
      {(void**)&p.pilot, P * p.K * B * sizeof(float)},
      {(void**)&p.pilot_c, P * p.K * sizeof(float)},
      {(void**)&p.pilot_s, P * p.K * sizeof(float)},
      {(void**)&p.mu0, P * B * sizeof(float2)},
      {(void**)&p.mu0f, P * B * sizeof(float)},
      {(void**)&p.vf, P * B * sizeof(float)},
      {(void**)&p.zt, P * B * sizeof(float2)},
      {(void**)&p.tprev, P * B * sizeof(float2)},
      {(void**)&p.muk, P * B * sizeof(float2)},
      {(void**)&p.S, P * B * B * sizeof(double)},
      {(void**)&p.Linv, P * ((size_t)B * (B + 1) / 2) * sizeof(float2)},  // packed rows
      {(void**)&p.pscal, P * 4 * sizeof(float)},
      {(void**)&p.dscal, P * 4 * sizeof(double)},
      {(void**)&p.k1part, (size_t)k1u * K1E * sizeof(float2)},
      {(void**)&p.k3part, (size_t)k3u * K3E * sizeof(float)},
      {(void**)&p.status, P * sizeof(int)},
      {(void**)&p.q_words,
       pl->persistent ? (mf::kQueueHead + P + (size_t)n_lines * p.n_ct) * sizeof(int) : 0},
      {(void**)&p.q_groups, pl->persistent ? (2 * (size_t)n_lines + 1) * sizeof(int) : 0},
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
  p.lines = lines_d;
  e = cudaMemset(pl->ws, 0, total);
  if (e == cudaSuccess && pl->persistent) {
    // work queue: the first item of every group of a pass, S(0) S(1) X(0)
    // S(2) X(1) ... S(L-1) X(L-2) X(L-1) (solves of line l: Pl items; pixel
    // CTAs of line l: n_ct n_rb items), then the pass size
    std::vector<int> g(2 * (size_t)n_lines + 1);
    long long at = 0;
    for (int gi = 0; gi < 2 * n_lines; ++gi) {
      g[gi] = (int)at;
      const bool last = gi == 2 * n_lines - 1;
      if (gi == 0 || ((gi & 1) && !last)) at += p.Pl;
      else at += (long long)p.n_ct * pl->lines[last ? n_lines - 1 : gi / 2 - 1].n_rb;
    }
    g[2 * n_lines] = (int)at;
    if (at > INT32_MAX) e = cudaErrorInvalidValue;
    if (e == cudaSuccess)
      e = cudaMemcpy(const_cast<int*>(p.q_groups), g.data(), g.size() * sizeof(int),
                     cudaMemcpyHostToDevice);
    pl->q_bytes = (mf::kQueueHead + P + (size_t)n_lines * p.n_ct) * sizeof(int);
    p.q_wait_ns = (long long)env_int("MF_QUEUE_WAIT_MS", 2000) * 1000000LL;
    pl->smem_queue = std::max({pl->smem_pixel, pl->smem_sinit, pl->smem_siter});
  }
  if (e == cudaSuccess)
    e = cudaMallocHost(&pl->lines_pinned, (size_t)n_lines * sizeof(mf::LineInfo));
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&pl->lines_copied, cudaEventDisableTiming);
  if (e == cudaSuccess) e = set_attrs(pl);
  if (e == cudaSuccess && pl->persistent) {
    // one wave of the work-queue kernel (queried after its shared-memory
    // attribute is set)
    const int per_sm = mf::queue_ctas_per_sm(pl->nj, pl->smem_queue);
    if (per_sm < 1) e = cudaErrorInvalidConfiguration;
    pl->grid_queue = per_sm * pl->num_sms;
  }
  if (e != cudaSuccess) {
    cudaFree(pl->ws);
    if (pl->lines_pinned) cudaFreeHost(pl->lines_pinned);
    if (pl->lines_copied) cudaEventDestroy(pl->lines_copied);
    delete pl;
    return fail(MF_ERR_CUDA, "plan set-up: %s", cudaGetErrorString(e));
  }
  *out = pl;
  return MF_OK;
}

// Upload the per-line lambda and iteration counts when they differ from the
// values on the device (the staging buffer is reused once its last copy ran).
mf_status upload_lines(mf_plan_s* pl, const double* lambda, const int32_t* n_iter,
                       cudaStream_t s) {
  bool same = pl->lines_valid;
  for (int l = 0; l < pl->n_lines && same; ++l)
    same = pl->lines[l].lambda == (float)lambda[l] && pl->lines[l].n_iter == n_iter[l];
  if (same) return MF_OK;
  for (int l = 0; l < pl->n_lines; ++l) {
    pl->lines[l].lambda = (float)lambda[l];
    pl->lines[l].n_iter = n_iter[l];
  }
  MF_CUDA(cudaEventSynchronize(pl->lines_copied));
  std::memcpy(pl->lines_pinned, pl->lines.data(), (size_t)pl->n_lines * sizeof(mf::LineInfo));
  MF_CUDA(cudaMemcpyAsync(const_cast<mf::LineInfo*>(pl->prm.lines), pl->lines_pinned,
                          (size_t)pl->n_lines * sizeof(mf::LineInfo), cudaMemcpyHostToDevice, s));
  MF_CUDA(cudaEventRecord(pl->lines_copied, s));
  pl->lines_valid = true;
  return MF_OK;
}

// Enqueue one retrieval of every line (lines with fewer iterations skip the
// later passes inside the kernels).
mf_status run_retrieval(mf_plan_s* pl, const float* cube, const float* k, double eps,
                        int32_t n_iter_max, const uint8_t* mask, const float* alpha_init,
                        float* alpha_out, float* albedo_out, cudaStream_t s,
                        const mf::Params* ck = nullptr) {
  if ((reinterpret_cast<uintptr_t>(cube) & 15) != 0)
    return fail(MF_ERR_INVALID_ARG, "cube must be 16-byte aligned");
  mf::Params p = pl->prm;
  p.cube = cube;
  p.k = k;
  p.mask = mask;
  p.alpha_init = alpha_init;
  p.alpha = alpha_out;
  p.albedo = albedo_out;
  p.eps = (float)eps;
  if (ck) {
    p.ck_alpha = ck->ck_alpha;
    p.ck_vec = ck->ck_vec;
    p.ck_sc = ck->ck_sc;
    p.ck_stages = ck->ck_stages;
    p.energy = ck->energy;
    p.energy_stride = ck->energy_stride;
  }
  const bool literal = (p.flags & MF_LITERAL) != 0;
  if (cube != pl->map_cube) {
    if (!encode_cube_map(&pl->map_stats, pl->prm, cube, 1, mf::kStatRows) ||
        !encode_cube_map(&pl->map_pixel, pl->prm, cube, mf::kTileCols, mf::kStageRows)) {
      pl->map_cube = nullptr;
      return fail(MF_ERR_CUDA, "cuTensorMapEncodeTiled failed for the cube");
    }
    pl->map_cube = cube;
  }
  auto enqueue = [&](cudaStream_t q) {
    pl->tl_kind.clear();
    cudaMemsetAsync(p.status, 0, (size_t)p.P * sizeof(int), q);
    if (pl->persistent) {
      // the statistics pass, then everything else in one launch
      cudaMemsetAsync(p.q_words, 0, pl->q_bytes, q);
      stats_dispatch(pl, p, mf::STAT_INIT, 0, q);
      queue_dispatch(pl, p, n_iter_max, q);
      return;
    }
    stats_dispatch(pl, p, mf::STAT_INIT, 0, q);
    solve_init_dispatch(pl, p, q);
    pixel_dispatch(pl, p, mf::PIX_INIT, n_iter_max > 0, 0, q);
    for (int it = 1; it <= n_iter_max; ++it) {
      if (literal) {
        solve_iter_dispatch(pl, p, mf::SOLVE_MEAN_ONLY, it, q);
        stats_dispatch(pl, p, mf::STAT_LITERAL, it, q);
        solve_literal_dispatch(pl, p, it, q);
      } else {
        solve_iter_dispatch(pl, p, mf::SOLVE_FUSED, it, q);
      }
      pixel_dispatch(pl, p, mf::PIX_ITER, it < n_iter_max, it, q);
    }
  };
  // direct launches when profiling (events per kernel) or when the caller is
  // capturing its own graph; otherwise one graph launch
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  MF_CUDA(cudaStreamIsCapturing(s, &cs));
  if (pl->profile || !pl->use_graph || ck || cs != cudaStreamCaptureStatusNone) {
    enqueue(s);
    if (p.energy) mf::energy_final_launch(s, p, n_iter_max);
    MF_CUDA(cudaGetLastError());
  } else {
    const mf_plan_s::GraphKey key{{cube, k, mask, alpha_init, alpha_out, albedo_out},
                                  n_iter_max, (float)eps, pl->timeline};
    int gi = -1;
    for (int i = 0; i < mf_plan_s::kGraphs; ++i)
      if (pl->gexec[i] && key == pl->gkey[i]) gi = i;
    if (gi < 0) {
      gi = pl->gnext;
      pl->gnext = (pl->gnext + 1) % mf_plan_s::kGraphs;
      if (pl->gexec[gi]) {
        MF_CUDA(cudaGraphExecDestroy(pl->gexec[gi]));
        pl->gexec[gi] = nullptr;
      }
      if (!pl->cap_stream) MF_CUDA(cudaStreamCreateWithFlags(&pl->cap_stream, cudaStreamNonBlocking));
      cudaGraph_t g = nullptr;
      MF_CUDA(cudaStreamBeginCapture(pl->cap_stream, cudaStreamCaptureModeThreadLocal));
      enqueue(pl->cap_stream);
      const cudaError_t e1 = cudaStreamEndCapture(pl->cap_stream, &g);
      if (e1 != cudaSuccess) return fail(MF_ERR_CUDA, "graph capture: %s", cudaGetErrorString(e1));
      const cudaError_t e2 = cudaGraphInstantiate(&pl->gexec[gi], g, 0);
      cudaGraphDestroy(g);
      if (e2 != cudaSuccess) {
        pl->gexec[gi] = nullptr;
        return fail(MF_ERR_CUDA, "graph instantiation: %s", cudaGetErrorString(e2));
      }
      pl->gkey[gi] = key;
    }
    MF_CUDA(cudaGraphLaunch(pl->gexec[gi], s));
  }
  pl->last_stream = s;
  return MF_OK;
}

mf_status check_scalars(double lambda, double eps, int32_t n_iter) {
  if (n_iter < 0 || n_iter > 100000) return fail(MF_ERR_INVALID_ARG, "n_iter = %d", n_iter);
  if (!std::isfinite(lambda) || !std::isfinite(eps))
    return fail(MF_ERR_NONFINITE_INPUT, "lambda or eps not finite");
  if (lambda < 0.0 || !(eps > 0.0))
    return fail(MF_ERR_INVALID_ARG, "need lambda >= 0 and eps > 0");
  return MF_OK;
}

}  // namespace

extern "C" {

mf_status mf_plan(const mf_desc* d, mf_plan_t* out) {
  g_last_error.clear();
  if (!d || !out) return fail(MF_ERR_INVALID_ARG, "null descriptor or output");
  const int64_t rows = d->rows;
  return build_plan(d, &rows, 1, nullptr, out);
}

mf_status mf_plan_ex(const mf_desc* d, const int64_t* line_rows, int32_t n_lines,
                     const mf_tuning* tuning, mf_plan_t* out) {
  g_last_error.clear();
  if (!d || !out) return fail(MF_ERR_INVALID_ARG, "null descriptor or output");
  const int64_t rows = d->rows;
  if (!line_rows) return build_plan(d, &rows, 1, tuning, out);
  return build_plan(d, line_rows, n_lines, tuning, out);
}

mf_status mf_plan_batched(const mf_desc* d, const int64_t* line_rows, int32_t n_lines,
                          mf_plan_t* out) {
  g_last_error.clear();
  if (!line_rows) return fail(MF_ERR_INVALID_ARG, "null line_rows");
  return build_plan(d, line_rows, n_lines, nullptr, out);
}

int32_t mf_num_lines(mf_plan_t pl) { return pl ? pl->n_lines : -1; }

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
  if (pl->lines_pinned) cudaFreeHost(pl->lines_pinned);
  if (pl->lines_copied) cudaEventDestroy(pl->lines_copied);
  for (auto& g : pl->gexec)
    if (g) cudaGraphExecDestroy(g);
  for (int b = 0; b < 2; ++b) {
    cudaFree(pl->a_cube[b]);
    cudaFree(pl->a_mask[b]);
    cudaFree(pl->a_k[b]);
    cudaFree(pl->a_alpha[b]);
    if (pl->copied[b]) cudaEventDestroy(pl->copied[b]);
    if (pl->consumed[b]) cudaEventDestroy(pl->consumed[b]);
  }
  if (pl->copy_stream) cudaStreamDestroy(pl->copy_stream);
  if (pl->cap_stream) cudaStreamDestroy(pl->cap_stream);
  cudaFree(pl->tl_dev);
  delete pl;
}

int64_t mf_num_partitions(mf_plan_t pl) { return pl ? pl->prm.P : -1; }

mf_status mf_retrieve(mf_plan_t pl, const float* cube, const float* k, double lambda, double eps,
                      int32_t n_iter, const uint8_t* mask, const float* alpha_init,
                      float* alpha_out, float* albedo_out, void* stream) {
  g_last_error.clear();
  if (!pl) return fail(MF_ERR_INVALID_ARG, "null plan");
  if (!cube || !k || !alpha_out) return fail(MF_ERR_INVALID_ARG, "null cube, k or alpha_out");
  if (pl->n_lines != 1)
    return fail(MF_ERR_INVALID_ARG, "plan of %d lines: use mf_retrieve_batched", pl->n_lines);
  mf_status st = check_scalars(lambda, eps, n_iter);
  if (st != MF_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  st = upload_lines(pl, &lambda, &n_iter, s);
  if (st != MF_OK) return st;
  return run_retrieval(pl, cube, k, eps, n_iter, mask, alpha_init, alpha_out, albedo_out, s);
}

mf_status mf_retrieve_energy(mf_plan_t pl, const float* cube, const float* k, double lambda,
                             double eps, int32_t n_iter, const uint8_t* mask, float* alpha_out,
                             double* energy_out, void* stream) {
  g_last_error.clear();
  if (!pl) return fail(MF_ERR_INVALID_ARG, "null plan");
  if (!cube || !k || !alpha_out || !energy_out)
    return fail(MF_ERR_INVALID_ARG, "null cube, k, alpha_out or energy_out");
  if ((reinterpret_cast<uintptr_t>(energy_out) & 7) != 0)
    return fail(MF_ERR_INVALID_ARG, "energy_out must be 8-byte aligned");
  if (pl->n_lines != 1) return fail(MF_ERR_UNSUPPORTED, "the energy output takes one line");
  if (pl->prm.flags & MF_LITERAL)
    return fail(MF_ERR_UNSUPPORTED, "the energy output follows the fused schedule (no MF_LITERAL)");
  mf_status st = check_scalars(lambda, eps, n_iter);
  if (st != MF_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  st = upload_lines(pl, &lambda, &n_iter, s);
  if (st != MF_OK) return st;
  mf::Params extra{};
  extra.energy = energy_out;
  extra.energy_stride = n_iter + 1;
  return run_retrieval(pl, cube, k, eps, n_iter, mask, nullptr, alpha_out, nullptr, s, &extra);
}

mf_status mf_retrieve_batched(mf_plan_t pl, const float* cube, const float* k,
                              const double* lambda, double eps, const int32_t* n_iter,
                              const uint8_t* mask, float* alpha_out, void* stream) {
  g_last_error.clear();
  if (!pl) return fail(MF_ERR_INVALID_ARG, "null plan");
  if (!cube || !k || !alpha_out || !lambda || !n_iter)
    return fail(MF_ERR_INVALID_ARG, "null cube, k, lambda, n_iter or alpha_out");
  int32_t n_max = 0;
  for (int l = 0; l < pl->n_lines; ++l) {
    mf_status st = check_scalars(lambda[l], eps, n_iter[l]);
    if (st != MF_OK) return st;
    n_max = std::max(n_max, n_iter[l]);
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  mf_status st = upload_lines(pl, lambda, n_iter, s);
  if (st != MF_OK) return st;
  return run_retrieval(pl, cube, k, eps, n_max, mask, nullptr, alpha_out, nullptr, s);
}

}  // extern "C"

namespace {

// Layout of a training checkpoint (caller-owned device memory): the forward's
// checkpoints and every buffer of the backward pass.
struct CkLayout {
  size_t alpha, vec, sc, abar0, abar1, rbar, coef, vkf, zf, bpart, psc, carry, mubar0, sbar,
      lbar, mu0bar, total;
};
CkLayout ck_layout(const mf_plan_s* pl, int n_iter, bool cube_grad) {
  const mf::Params& p = pl->prm;
  const size_t P = p.P, B = p.B, S = (size_t)n_iter + 1;
  const size_t npix = (size_t)p.rows * p.cols;
  const size_t units = (size_t)p.cols * pl->lines[0].n_rb;
  CkLayout L{};
  size_t off = 0;
  auto take = [&](size_t bytes) {
    off = align_up(off, 256);
    const size_t at = off;
    off += bytes;
    return at;
  };
  L.alpha = take(S * npix * sizeof(float));
  L.vec = take(P * S * 4 * B * sizeof(float2));
  L.sc = take(P * S * 4 * sizeof(double));
  L.abar0 = take(npix * sizeof(float));
  L.abar1 = take(npix * sizeof(float));
  L.rbar = take(npix * sizeof(float));
  L.coef = take(cube_grad ? S * npix * 2 * sizeof(float) : 0);
  L.vkf = take(P * B * sizeof(float));
  L.zf = take(P * S * B * sizeof(float));
  L.bpart = take(units * mf::bwd_entries((int)B) * sizeof(float));
  L.psc = take(P * mf::kPsc * sizeof(double));
  L.carry = take(P * B * sizeof(float2));
  L.mubar0 = take(P * B * sizeof(float2));
  L.sbar = take(P * B * sizeof(double));
  L.lbar = take(P * sizeof(double));
  L.mu0bar = take(P * B * sizeof(float));
  L.total = align_up(off, 256);
  return L;
}

}  // namespace

extern "C" {

size_t mf_ckpt_bytes(mf_plan_t pl, int32_t n_iter, int32_t cube_grad) {
  if (!pl || n_iter < 0) return 0;
  return ck_layout(pl, n_iter, cube_grad != 0).total;
}

mf_status mf_retrieve_train(mf_plan_t pl, const float* cube, const float* k, double lambda,
                            double eps, int32_t n_iter, const uint8_t* mask, float* alpha_out,
                            void* ckpt, int32_t cube_grad, void* stream) {
  g_last_error.clear();
  if (!pl) return fail(MF_ERR_INVALID_ARG, "null plan");
  if (!cube || !k || !alpha_out || !ckpt)
    return fail(MF_ERR_INVALID_ARG, "null cube, k, alpha_out or ckpt");
  if (pl->n_lines != 1) return fail(MF_ERR_UNSUPPORTED, "the backward pass takes one line");
  if (pl->prm.flags & MF_LITERAL)
    return fail(MF_ERR_UNSUPPORTED, "the backward pass follows the fused schedule (no MF_LITERAL)");
  if ((reinterpret_cast<uintptr_t>(ckpt) & 255) != 0)
    return fail(MF_ERR_INVALID_ARG, "ckpt must be 256-byte aligned");
  mf_status st = check_scalars(lambda, eps, n_iter);
  if (st != MF_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  st = upload_lines(pl, &lambda, &n_iter, s);
  if (st != MF_OK) return st;
  const CkLayout L = ck_layout(pl, n_iter, cube_grad != 0);
  char* base = static_cast<char*>(ckpt);
  mf::Params ck{};
  ck.ck_alpha = reinterpret_cast<float*>(base + L.alpha);
  ck.ck_vec = reinterpret_cast<float2*>(base + L.vec);
  ck.ck_sc = reinterpret_cast<double*>(base + L.sc);
  ck.ck_stages = n_iter + 1;
  st = run_retrieval(pl, cube, k, eps, n_iter, mask, nullptr, alpha_out, nullptr, s, &ck);
  if (st != MF_OK) return st;
  pl->train.ckpt = ckpt;
  pl->train.n_iter = n_iter;
  pl->train.cube_grad = cube_grad != 0;
  pl->train.cube = cube;
  pl->train.k = k;
  pl->train.mask = mask;
  pl->train.eps = eps;
  return MF_OK;
}

mf_status mf_retrieve_backward(mf_plan_t pl, const void* ckpt, const float* grad_alpha,
                               float* grad_k, float* grad_lambda, float* grad_cube,
                               void* stream) {
  g_last_error.clear();
  if (!pl || !ckpt || !grad_alpha || !grad_k || !grad_lambda)
    return fail(MF_ERR_INVALID_ARG, "null plan, ckpt, grad_alpha, grad_k or grad_lambda");
  if (ckpt != pl->train.ckpt)
    return fail(MF_ERR_INVALID_ARG, "ckpt does not hold this plan's last mf_retrieve_train");
  if (grad_cube && !pl->train.cube_grad)
    return fail(MF_ERR_INVALID_ARG, "the forward was checkpointed without the cube gradient");
  const int n = pl->train.n_iter;
  const CkLayout L = ck_layout(pl, n, pl->train.cube_grad);
  char* base = static_cast<char*>(const_cast<void*>(ckpt));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  mf::Params p = pl->prm;
  p.cube = pl->train.cube;
  p.k = pl->train.k;
  p.mask = pl->train.mask;
  p.eps = (float)pl->train.eps;
  p.ck_alpha = reinterpret_cast<float*>(base + L.alpha);
  p.ck_vec = reinterpret_cast<float2*>(base + L.vec);
  p.ck_sc = reinterpret_cast<double*>(base + L.sc);
  p.ck_stages = n + 1;
  mf::BwdParams b{};
  b.n_iter = n;
  b.grad_alpha = grad_alpha;
  b.abar[0] = reinterpret_cast<float*>(base + L.abar0);
  b.abar[1] = reinterpret_cast<float*>(base + L.abar1);
  b.rbar = reinterpret_cast<float*>(base + L.rbar);
  b.coef = grad_cube ? reinterpret_cast<float*>(base + L.coef) : nullptr;
  b.grad_cube = grad_cube;
  b.vkf = reinterpret_cast<float*>(base + L.vkf);
  b.zf = reinterpret_cast<float*>(base + L.zf);
  b.bpart = reinterpret_cast<float*>(base + L.bpart);
  b.psc = reinterpret_cast<double*>(base + L.psc);
  b.carry = reinterpret_cast<float2*>(base + L.carry);
  b.mubar0 = reinterpret_cast<float2*>(base + L.mubar0);
  b.sbar = reinterpret_cast<double*>(base + L.sbar);
  b.lbar = reinterpret_cast<double*>(base + L.lbar);
  b.mu0bar_n = reinterpret_cast<float*>(base + L.mu0bar);
  b.grad_k = grad_k;
  b.grad_lambda = grad_lambda;
  if (p.cube != pl->map_cube) {
    if (!encode_cube_map(&pl->map_stats, pl->prm, p.cube, 1, mf::kStatRows) ||
        !encode_cube_map(&pl->map_pixel, pl->prm, p.cube, mf::kTileCols, mf::kStageRows)) {
      pl->map_cube = nullptr;
      return fail(MF_ERR_CUDA, "cuTensorMapEncodeTiled failed for the cube");
    }
    pl->map_cube = p.cube;
  }
  const size_t smem_px = mf::bwd_pixel_smem_bytes(p.B, pl->nj);
  const size_t smem_sv = mf::bwd_solve_smem_bytes(p.B);
  MF_CUDA(mf::bwd_set_attributes(pl->nj, smem_px, smem_sv));
  // zero the per-partition accumulators (psc, carry, mubar0, sbar, lbar)
  MF_CUDA(cudaMemsetAsync(base + L.psc, 0, L.mu0bar - L.psc, s));
  const int grid_px = p.n_ct * pl->lines[0].n_rb;
  for (int k = n; k >= 0; --k)
    mf::bwd_launch_stage(pl->nj, grid_px, smem_px, smem_sv, s, pl->map_pixel, p, b, k);
  mf::bwd_launch_final(pl->nj, smem_px, s, p, b);
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

mf_status mf_retrieve_host_async(mf_plan_t pl, const float* cube, const float* k, double lambda,
                                 double eps, int32_t n_iter, const uint8_t* mask,
                                 float* alpha_out, void* stream) {
  g_last_error.clear();
  if (!pl || !cube || !k || !alpha_out) return fail(MF_ERR_INVALID_ARG, "null argument");
  const mf::Params& g = pl->prm;
  const size_t npix = (size_t)g.rows * g.cols;
  const size_t cube_bytes = npix * g.bands_total * sizeof(float);
  if (!pl->copy_stream) {
    for (int b = 0; b < 2; ++b) {
      MF_CUDA(cudaMalloc(&pl->a_cube[b], cube_bytes));
      MF_CUDA(cudaMalloc(&pl->a_mask[b], npix));
      MF_CUDA(cudaMalloc(&pl->a_k[b], (size_t)g.B * sizeof(float)));
      MF_CUDA(cudaMalloc(&pl->a_alpha[b], npix * sizeof(float)));
      MF_CUDA(cudaEventCreateWithFlags(&pl->copied[b], cudaEventDisableTiming));
      MF_CUDA(cudaEventCreateWithFlags(&pl->consumed[b], cudaEventDisableTiming));
    }
    MF_CUDA(cudaStreamCreateWithFlags(&pl->copy_stream, cudaStreamNonBlocking));
  }
  const int b = pl->aslot;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // slot b's buffers are free once the retrieval that last used them and
  // its copy of alpha out are done (an event never recorded: no wait)
  MF_CUDA(cudaStreamWaitEvent(pl->copy_stream, pl->consumed[b], 0));
  MF_CUDA(cudaMemcpyAsync(pl->a_cube[b], cube, cube_bytes, cudaMemcpyHostToDevice, pl->copy_stream));
  MF_CUDA(cudaMemcpyAsync(pl->a_k[b], k, (size_t)g.B * sizeof(float), cudaMemcpyHostToDevice,
                          pl->copy_stream));
  if (mask)
    MF_CUDA(cudaMemcpyAsync(pl->a_mask[b], mask, npix, cudaMemcpyHostToDevice, pl->copy_stream));
  MF_CUDA(cudaEventRecord(pl->copied[b], pl->copy_stream));
  MF_CUDA(cudaStreamWaitEvent(s, pl->copied[b], 0));
  mf_status st = mf_retrieve(pl, pl->a_cube[b], pl->a_k[b], lambda, eps, n_iter,
                             mask ? pl->a_mask[b] : nullptr, nullptr, pl->a_alpha[b], nullptr,
                             stream);
  if (st != MF_OK) return st;
  MF_CUDA(cudaMemcpyAsync(alpha_out, pl->a_alpha[b], npix * sizeof(float), cudaMemcpyDeviceToHost,
                          s));
  MF_CUDA(cudaEventRecord(pl->consumed[b], s));
  pl->aslot = b ^ 1;
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

mf_status mf_timeline(mf_plan_t pl, int32_t enable) {
  g_last_error.clear();
  if (!pl) return fail(MF_ERR_INVALID_ARG, "null plan");
  if (enable && !pl->tl_dev) {
    const cudaError_t e = cudaMalloc(&pl->tl_dev, 2 * kMaxSpans * sizeof(unsigned long long));
    if (e != cudaSuccess) {
      pl->tl_dev = nullptr;
      return fail(e == cudaErrorMemoryAllocation ? MF_ERR_OOM : MF_ERR_CUDA,
                  "timeline buffer: %s", cudaGetErrorString(e));
    }
    MF_CUDA(cudaMemset(pl->tl_dev, 0, 2 * kMaxSpans * sizeof(unsigned long long)));
    MF_CUDA(cudaDeviceSynchronize());
  }
  pl->timeline = enable != 0;
  return MF_OK;
}

mf_status mf_timeline_read(mf_plan_t pl, double* start_us, double* end_us, int32_t* kind,
                           int32_t cap, int32_t* n) {
  g_last_error.clear();
  if (!pl || !start_us || !end_us || !kind || !n || cap < 0)
    return fail(MF_ERR_INVALID_ARG, "bad argument");
  *n = 0;
  if (!pl->tl_dev) return MF_OK;
  if (pl->last_stream) MF_CUDA(cudaStreamSynchronize(pl->last_stream));
  const size_t m = pl->tl_kind.size();
  std::vector<unsigned long long> w(2 * std::max<size_t>(m, 1));
  if (m) MF_CUDA(cudaMemcpy(w.data(), pl->tl_dev, 2 * m * sizeof(unsigned long long),
                            cudaMemcpyDeviceToHost));
  // cleared for the next retrieval, whatever stream it runs on
  MF_CUDA(cudaMemset(pl->tl_dev, 0, 2 * kMaxSpans * sizeof(unsigned long long)));
  MF_CUDA(cudaDeviceSynchronize());
  // times relative to the earliest recorded start; a slot whose launch
  // recorded nothing (no CTA ran, e.g. a line with its iterations done) is
  // reported with start = end = -1
  unsigned long long t0 = ~0ull;
  for (size_t i = 0; i < m; ++i)
    if (w[2 * i + 1]) t0 = std::min(t0, ~w[2 * i]);
  const int32_t out = (int32_t)std::min<size_t>(m, (size_t)cap);
  for (int32_t i = 0; i < out; ++i) {
    kind[i] = pl->tl_kind[i];
    if (w[2 * i + 1]) {
      start_us[i] = (double)(~w[2 * i] - t0) * 1e-3;
      end_us[i] = (double)(w[2 * i + 1] - t0) * 1e-3;
    } else {
      start_us[i] = end_us[i] = -1.0;
    }
  }
  *n = out;
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
  if (pl->persistent) {
    // a work-queue retrieval that stopped early leaves items undone: every
    // partition is suspect
    int abort_word = 0;
    MF_CUDA(cudaMemcpy(&abort_word, pl->prm.q_words + 2, sizeof(int), cudaMemcpyDeviceToHost));
    if (abort_word != 0)
      for (int i = 0; i < pl->prm.P; ++i)
        if (status[i] == MF_OK) status[i] = MF_ERR_TIMEOUT;
  }
  for (int i = 0; i < pl->prm.P; ++i)
    if (status[i] != MF_OK) return (mf_status)status[i];
  return MF_OK;
}

}  // extern "C"
