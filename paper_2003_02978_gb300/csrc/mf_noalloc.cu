// mf_background_noalloc: the initial background statistics (mean and
// covariance of every partition) for callers that cannot allocate device
// memory.
//
// Some callers of this library may not allocate device memory once they are
// running: real-time flight or ground-segment pipelines that forbid any
// allocation after start-up, and hosts whose device memory is owned by
// another allocator (a framework's caching pool, an embedded runtime) that
// this library cannot call.  They cannot create a plan (mf_plan allocates its
// workspace), so this entry point keeps the per-block partial moments in a
// fixed file-scope device array instead.
//
// That array is a __device__ global: every GPU that loads the library holds
// its kNoAllocScratchBytes (64 MiB) until the process exits.  In host code
// its name is only a host-side stand-in, not a device address, so the first
// call on each device looks up the device address with cudaGetSymbolAddress
// (with that device current) and caches it, together with the kernels'
// shared-memory limits; make that first call before any stream capture.  The
// cached address belongs to the device's primary context: a process that
// resets the device (cudaDeviceReset) must not call this entry point again.
// Every call shares the array and leaves the last call's contents behind:
// each call rewrites the line table and clears the status words (what must
// start at zero), and calls that overlap on the GPU (different streams, or
// several host threads) race on it.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <mutex>
#include <string>

#include "../../include/mf.h"
#include "mf_common.cuh"

namespace {

constexpr size_t kNoAllocScratchBytes = 64ull << 20;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

struct DeviceScratch {
  bool ready = false;
  unsigned char* ptr = nullptr;  // device address of g_noalloc_scratch
};
std::mutex g_mutex;
DeviceScratch g_devices[kMaxDevices];
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;  // set under g_mutex

// the line table of one call, written by the device from a kernel argument
// (no host staging buffer whose lifetime the copy would depend on)
__global__ void write_line_kernel(mf::LineInfo* dst, mf::LineInfo line) { *dst = line; }

mf_status fail(mf_status s, const std::string& msg) {
  mf::set_last_error(msg);
  return s;
}

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

int nj_bucket(int B4) {
  const int need = (B4 + 1) / 2;
  const int buckets[] = {1, 2, 4, 6, 8, 9, 10, 12, 16};
  for (int b : buckets)
    if (b >= need) return b;
  return -1;
}

// once per device, with that device current: device address of the array and
// the kernels' shared-memory limits
mf_status setup_device(int dev, unsigned char** out) {
  std::lock_guard<std::mutex> lock(g_mutex);
  if (dev < 0 || dev >= kMaxDevices) return fail(MF_ERR_UNSUPPORTED, "device index out of range");
  if (!g_encode) {
    void* fp = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fp, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return fail(MF_ERR_CUDA, "cuTensorMapEncodeTiled is not available");
    g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fp);
  }
  DeviceScratch& d = g_devices[dev];
  if (!d.ready) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess)
      return fail(MF_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    const int bmax = mf::kMaxB, ba = mf::aug_width(bmax, mf::kMaxDirs);
    for (int nj : {1, 2, 4, 6, 8, 9, 10, 12, 16}) {
      e = mf::stats_set_attributes(nj, mf::stats_smem_bytes(8 * nj, mf::kDirsFp32));
      if (e != cudaSuccess) break;
    }
    if (e == cudaSuccess) e = mf::background_set_attributes(mf::background_smem_bytes(bmax, ba));
    if (e != cudaSuccess)
      return fail(MF_ERR_CUDA, std::string("kernel attributes: ") + cudaGetErrorString(e));
    d.ptr = static_cast<unsigned char*>(p);
    d.ready = true;
  }
  *out = d.ptr;
  return MF_OK;
}

// (after setup_device, which resolved g_encode)
bool encode_map(CUtensorMap* m, const mf::Params& p, const float* cube) {
  const PFN_cuTensorMapEncodeTiled_v12000 fn = g_encode;
  if (!fn) return false;
  const cuuint64_t dims[3] = {(cuuint64_t)p.bands_total, (cuuint64_t)p.cols, (cuuint64_t)p.rows};
  const cuuint64_t strides[2] = {(cuuint64_t)p.bands_total * sizeof(float),
                                 (cuuint64_t)p.bands_total * p.cols * sizeof(float)};
  const cuuint32_t box[3] = {(cuuint32_t)p.B, 1u, (cuuint32_t)mf::kStatRows};
  const cuuint32_t estr[3] = {1, 1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(cube), dims, strides, box,
            estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

extern "C" mf_status mf_background_noalloc(const mf_desc* d, const float* cube,
                                           const uint8_t* mask, double* mu0, double* cov0,
                                           void* stream) {
  mf::set_last_error("");
  if (!d || !cube || !mu0 || !cov0) return fail(MF_ERR_INVALID_ARG, "null argument");
  if (d->rows <= 0 || d->cols <= 0 || d->bands_total <= 0 || d->band_lo < 0 ||
      d->band_hi > d->bands_total || d->band_hi <= d->band_lo || d->col_group < 1)
    return fail(MF_ERR_INVALID_ARG, "bad shape, band window or col_group");
  if (d->layout != MF_BIP) return fail(MF_ERR_UNSUPPORTED, "only the BIP layout is supported");
  const int B = d->band_hi - d->band_lo;
  if (B < 8 || B > mf::kMaxB || B % 4 || d->band_lo % 4 || d->bands_total % 4)
    return fail(MF_ERR_UNSUPPORTED, "need 8 <= B <= 128 and 16-byte aligned pixel windows");
  if (d->rows > (1LL << 30) || d->cols > (1LL << 24) || d->rows * d->cols > (1LL << 40))
    return fail(MF_ERR_UNSUPPORTED, "cube too large");
  if ((reinterpret_cast<uintptr_t>(cube) & 15) != 0)
    return fail(MF_ERR_INVALID_ARG, "cube must be 16-byte aligned");

  mf::Params p{};
  p.rows = (int)d->rows;
  p.cols = (int)d->cols;
  p.bands_total = (int)d->bands_total;
  p.band_lo = d->band_lo;
  p.B = B;
  p.B4 = B / 4;
  p.G = (int)std::min<int64_t>(d->col_group, d->cols);
  p.Pl = (p.cols + p.G - 1) / p.G;
  p.P = p.Pl;
  p.n_lines = 1;
  p.K = mf::kDirsFp32;
  p.BA = mf::aug_width(B, p.K);
  p.flags = d->flags;
  p.cube = cube;
  p.mask = mask;

  // scratch layout: line table (1) | directions (P, K, B), offsets (P, K),
  // scales (P, K) float | status (P) int | moments
  const size_t P = (size_t)p.P;
  const size_t K1E = (size_t)mf::k1_entries(p.BA);
  const size_t line_bytes = align256(sizeof(mf::LineInfo));
  const size_t dir_bytes = align256(P * p.K * B * sizeof(float));
  const size_t off_bytes = align256(P * p.K * sizeof(float));
  const size_t fixed = line_bytes + dir_bytes + 2 * off_bytes + align256(P * sizeof(int));
  const size_t per_chunk = P * p.G * K1E * sizeof(float2);  // one row chunk per column
  if (fixed + per_chunk > kNoAllocScratchBytes) {
    char msg[256];
    snprintf(msg, sizeof msg,
             "%zu partitions of %d bands need %zu bytes of scratch; the fixed array holds %zu",
             P, B, fixed + per_chunk, kNoAllocScratchBytes);
    return fail(MF_ERR_UNSUPPORTED, msg);
  }
  // as many row chunks per column as fit (more CTAs), at most the plan's choice
  long nsc = std::max<long>(1, (2400 + p.cols - 1) / p.cols);
  nsc = std::min<long>(nsc, (long)((kNoAllocScratchBytes - fixed) / per_chunk));
  int sc = (int)((p.rows + nsc - 1) / nsc);
  sc = std::max(mf::kStatRows, (sc + mf::kStatRows - 1) / mf::kStatRows * mf::kStatRows);
  mf::LineInfo line{};
  line.rows = p.rows;
  line.sc_rows = sc;
  line.n_sc = (p.rows + sc - 1) / sc;
  p.n_items = p.cols * line.n_sc;
  p.line0 = line;

  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(MF_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  unsigned char* base = nullptr;
  mf_status st = setup_device(dev, &base);
  if (st != MF_OK) return st;
  p.lines = reinterpret_cast<const mf::LineInfo*>(base);
  p.pilot = reinterpret_cast<float*>(base + line_bytes);
  p.pilot_c = reinterpret_cast<float*>(base + line_bytes + dir_bytes);
  p.pilot_s = reinterpret_cast<float*>(base + line_bytes + dir_bytes + off_bytes);
  p.status = reinterpret_cast<int*>(base + line_bytes + dir_bytes + 2 * off_bytes);
  p.k1part = reinterpret_cast<float2*>(base + fixed);

  CUtensorMap map;
  if (!encode_map(&map, p, cube)) return fail(MF_ERR_CUDA, "cuTensorMapEncodeTiled failed");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  write_line_kernel<<<1, 1, 0, s>>>(reinterpret_cast<mf::LineInfo*>(base), line);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemsetAsync(p.status, 0, P * sizeof(int), s);
  if (e != cudaSuccess) return fail(MF_ERR_CUDA, std::string("set-up copies: ") + cudaGetErrorString(e));
  const int nj = nj_bucket(p.B4);
  mf::pilot_dirs_launch(s, p);
  mf::stats_launch(nj, p.n_items, mf::stats_smem_bytes(B, p.K), s, map, p, mf::STAT_INIT, 0);
  mf::background_launch(mf::background_smem_bytes(B, p.BA), s, p, mu0, cov0);
  e = cudaGetLastError();
  if (e != cudaSuccess) return fail(MF_ERR_CUDA, std::string("launch: ") + cudaGetErrorString(e));
  return MF_OK;
}
