// Statistics kernel on the tensor cores (precision form MF_BF16SPLIT).
//
// Same quantity as the float32 statistics kernel: the augmented second
// moments G = sum_i u_i u_i^T of u_i = [e_i, a_i, b_i, 1] (residual of the
// albedo-direction split, Sec. II-C; see mf_stats.cu), per partition and
// chunk of rows, which the solve kernels turn into C^0 (Fig. 1) or C^k
// (Eq. (11), literal schedule).
//
// Each u_i (float32) is split into bf16 hi + lo (hi = bf16(u), lo =
// bf16(u - hi)), so that u = hi + lo to about 2^-18 relative, and
//   G = H^T H + H^T L + L^T H + L^T L.
// (L^T L is small per product but biased on the diagonal; without it C^0
// is off by ~1e-5 relative and alpha by ~2e-4.)  Since G is symmetric,
// L^T H = (H^T L)^T, so two tcgen05.mma kind::f16 per 16 pixels suffice:
//   D[:, 0 : 2 NP]  = H^T [H | L]       (M = 128, N = 2 NP)
//   D[:, 0 : NP]   += L^T L             (M = 128, N = NP)
// where NP = B + 4 rounded up to 16; an operand set holds H and L side by
// side along N (MN-major core matrices), followed by 128 - NP zero columns,
// and an A operand is the first 128 columns from H's or L's start (the
// columns past NP give rows of D that the epilogue ignores).  D accumulates in float32 in tensor memory;
// the epilogue forms Q = (H^T H + L^T L) / 2 + H^T L, and G = Q + Q^T is
// completed where the per-item moments are summed (each item's Q is stored
// column-major, BA x BA floats, so that the stores of a warp are
// contiguous).
//
// Persistent, warp-specialised kernel: one CTA per SM walks work items
// (detector column, chunk of at most 1024 rows) of 128-pixel stages, with
// hand-offs on shared-memory mbarriers only:
//   warp 8 (producer): TMA box of 128 rows x B bands (float32) -> one of
//            three float32 stages (two for the widest windows)
//   warps 0-7 (converters, a lane pair per pixel): albedo split,
//            augmentation, bf16 hi/lo into MN-major core matrices of one of
//            two operand sets
//   warp 9 (issuer, one lane): 8 x 2 MMAs (K = 16 pixels each) per stage into
//            one of two tensor-memory accumulators (alternating per stage);
//            tcgen05.commit frees the operand set and publishes the stage
//   warps 10-13 (epilogue): tcgen05.ld of a finished stage accumulator, added
//            into the item's running sum in tensor memory; after the item's
//            last stage its moments are written as float pairs.
// The reference direction of each partition (the mean of its first few
// valid pixels, or mu^0) comes from global memory (pilot_kernel below for
// the initialisation).
#include "mf_common.cuh"
#include "mf_pixel_io.cuh"
#include "mf_tc.cuh"
#include "mf_tma.cuh"
#include "../../include/mf.h"

#include <cuda_bf16.h>

namespace mf {

namespace {
constexpr int kTcThreads = 448;     // 8 converter warps, producer, issuer, 4 epilogue warps
constexpr int kTcConv = 256;        // converter threads (warps 0-7)
constexpr int kTcRows = 128;          // pixels per stage (K of one stage)
constexpr int kTcM = 128;             // MMA M (rows of G, >= B + 4)
constexpr uint32_t kTmemCols = 512;   // two stage accumulators (2 NP each) and a running sum (NP)

constexpr int kMaxFpStages = 3;

struct TcSmem {
  int NP;                  // N: augmented width rounded up to 16
  int nfp;                 // float32 stages in flight (3, or 2 for wide windows)
  size_t opb;              // one operand set: 16 K groups of [H | L | zeros]
  size_t kstride;          // bytes between core matrices along K (8 pixels)
  size_t lo_off;           // L's first core matrix relative to H's
  size_t pad_off, pad_bytes;  // zero columns after L in each K group
  int accw;                // tensor-memory columns of one stage accumulator (2 NP, 32-aligned)
  size_t stage_bytes;      // float32 stage: 128 rows x B
  size_t ops_off, stage_off, ref_off, bar_off, slot_off, total;
};
__host__ __device__ inline TcSmem tc_layout_n(int B, int nfp) {
  TcSmem L;
  const int BA = (B + 6) / 4 * 4;
  L.NP = (BA + 15) / 16 * 16;
  L.nfp = nfp;
  L.accw = (2 * L.NP + 31) / 32 * 32;  // accumulators at 0 and accw, running sum at 2 accw
  L.lo_off = (size_t)(L.NP / 8) * 128;
  // an A operand is 128 columns (M) from H's or L's start: from L's start it
  // runs 128 - NP columns past L, into zero columns that close the K group,
  // so that every operand byte the tensor core reads is written data
  L.pad_off = 2 * L.lo_off;
  L.pad_bytes = (size_t)((kTcM - L.NP) / 8) * 128;
  L.kstride = L.pad_off + L.pad_bytes;
  L.opb = L.kstride * (kTcRows / 8);
  L.stage_bytes = (size_t)kTcRows * B * sizeof(float);
  // two operand sets, then the float32 stages
  L.ops_off = 0;
  L.stage_off = L.ops_off + 2 * L.opb;
  L.ref_off = L.stage_off + nfp * L.stage_bytes;
  L.bar_off = L.ref_off + 2 * (size_t)(kMaxB + 4) * sizeof(float);
  L.slot_off = L.bar_off + 24 * sizeof(uint64_t);
  L.total = L.slot_off + 16;
  return L;
}
__host__ __device__ inline TcSmem tc_layout(int B) {
  TcSmem L = tc_layout_n(B, kMaxFpStages);
  if (L.total + 1024 > 227 * 1024) L = tc_layout_n(B, 2);
  return L;
}

__device__ __forceinline__ uint32_t bf162_bits(__nv_bfloat162 v) {
  return *reinterpret_cast<const uint32_t*>(&v);
}
// bf16 hi and lo parts of 4 values, packed pairwise: hi = bf16(v) (round to
// nearest), lo = bf16(v - hi), v - hi exact in float32
__device__ __forceinline__ void split_bf16x4(float4 v, uint2& hi, uint2& lo) {
  const float2 v01 = make_float2(v.x, v.y), v23 = make_float2(v.z, v.w);
  const __nv_bfloat162 h01 = __float22bfloat162_rn(v01), h23 = __float22bfloat162_rn(v23);
  const float2 r01 = __ffma2_rn(__bfloat1622float2(h01), make_float2(-1.f, -1.f), v01);
  const float2 r23 = __ffma2_rn(__bfloat1622float2(h23), make_float2(-1.f, -1.f), v23);
  hi = make_uint2(bf162_bits(h01), bf162_bits(h23));
  lo = make_uint2(bf162_bits(__float22bfloat162_rn(r01)), bf162_bits(__float22bfloat162_rn(r23)));
}
}  // namespace

size_t stats_tc_smem_bytes(int B) { return tc_layout(B).total + 1024; }
// 64 <= B <= 92.  B >= 64: with fewer bands the target is close to the albedo direction and
// the 2^-18 representation error of the two-term split is amplified beyond
// the stated bound (it also makes NP >= 80, so that an A operand, 128
// columns from H's start, stays inside its K group, and one from L's start
// ends inside the shared-memory allocation).  B <= 92: the two stage
// accumulators and the running sum fit the 512 tensor-memory columns.
bool stats_tc_supported(int B) {
  if (B < 64 || B + 4 > kTcM || stats_tc_smem_bytes(B) > 227 * 1024) return false;
  const TcSmem L = tc_layout(B);
  return 2 * L.accw + L.NP <= (int)kTmemCols;  // B <= 92
}

// Mean of the first (up to) kPilot valid pixels of every partition
// (row-major over its columns): the reference direction m of the initial
// statistics.  Any m gives the same moments in exact arithmetic; a mean of a
// few pixels rather than one leaves the augmented vectors [e, rho - 1, ..]
// closer to zero mean, so that the float32 sums cancel less.  One warp per
// partition.
constexpr int kPilot = 8;
__global__ void pilot_kernel(Params p) {
  // a retrieval's first kernel: the statistics kernel after it may start its
  // cube copies at once (its converters wait before reading the reference)
  pdl_trigger();
  const LaunchSpan span(p);
  const int part = blockIdx.x * 4 + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (part >= p.P) return;
  const LineInfo line = p.lines[part_line(p, part)];
  const int c0 = part_col0(p, part), ncp = part_ncols(p, part);
  const long total = (long)line.rows * ncp;
  float sum[kMaxB / 32] = {};  // bands lane + 32 q
  int n = 0;                   // warp-uniform
  for (long base = 0; base < total && n < kPilot; base += 32) {
    const long i = base + lane;
    bool ok = false;
    if (i < total) {
      const int row = line.row0 + (int)(i / ncp), col = c0 + (int)(i % ncp);
      ok = !p.mask || p.mask[(size_t)row * p.cols + col] == 0;
      if (ok) {
        const float4* px = reinterpret_cast<const float4*>(pixel_ptr(p, row, col));
        // every band finite (the loads are independent: no short circuit)
        for (int f = 0; f < p.B4; ++f) ok &= finite4(__ldg(px + f));
      }
    }
    unsigned bal = __ballot_sync(0xffffffffu, ok);
    // the batch's valid pixels (up to those still needed): all their loads
    // first, then the sum in pixel order
    float vals[kPilot][kMaxB / 32];
    int cnt = 0;
#pragma unroll
    for (int j = 0; j < kPilot; ++j) {
      if (bal && n + cnt < kPilot) {
        const long v = base + __ffs(bal) - 1;
        bal &= bal - 1;
        const float* px = pixel_ptr(p, line.row0 + (int)(v / ncp), c0 + (int)(v % ncp));
#pragma unroll
        for (int q = 0; q < kMaxB / 32; ++q)
          vals[j][q] = lane + 32 * q < p.B ? px[lane + 32 * q] : 0.f;
        ++cnt;
      }
    }
#pragma unroll
    for (int j = 0; j < kPilot; ++j)
      if (j < cnt)
#pragma unroll
        for (int q = 0; q < kMaxB / 32; ++q) sum[q] += vals[j][q];
    n += cnt;
  }
  const float inv = n > 0 ? 1.f / (float)n : 0.f;
  float n2 = 0.f;
#pragma unroll
  for (int q = 0; q < kMaxB / 32; ++q)
    if (lane + 32 * q < p.B) {
      const float m = sum[q] * inv;
      p.pilot[(size_t)part * p.B + lane + 32 * q] = m;
      n2 = fmaf(m, m, n2);
    }
  n2 = warp_sumf(n2);
  // one direction, offset 1: the coefficient a = rho - 1 of the split
  if (lane == 0) {
    p.pilot_c[part] = 1.f;
    p.pilot_s[part] = n2 > 0.f ? 1.f / n2 : 0.f;
  }
}

// named barrier 1 among the converter warps.  It follows code where only
// some lanes of a warp store (the next item's reference): the warp is
// reconverged first, and the barrier is the non-aligned form, which counts
// every thread however the warp arrives (the aligned bar.sync needs a
// converged warp, else the count can complete before every warp is in)
__device__ __forceinline__ void conv_bar() {
  __syncwarp();
  asm volatile("barrier.sync 1, %0;" ::"n"(kTcConv) : "memory");
}

template <int NJ>
__global__ void __launch_bounds__(kTcThreads, 1)
    stats_tc_kernel(const __grid_constant__ CUtensorMap map, Params p, int mode, int pass) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ int s_abort;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int B = p.B, B4 = p.B4, BA = p.BA;
  const TcSmem L = tc_layout(B);
  const int NP = L.NP;
  unsigned char* ops = smem_raw + L.ops_off;
  const int NF = L.nfp;
  float* stage_base = reinterpret_cast<float*>(smem_raw + L.stage_off);
  auto stage = [&](int q) { return stage_base + (size_t)q * (L.stage_bytes / sizeof(float)); };
  float* s_ref = reinterpret_cast<float*>(smem_raw + L.ref_off);  // [2][kMaxB + 4]
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw + L.bar_off);
  uint64_t* fp_full = bars;        // [NF] float32 stage landed (TMA)
  uint64_t* fp_empty = bars + 4;   // [NF] float32 stage read by every converter warp
  uint64_t* op_full = bars + 8;    // [2] operand set written by every converter warp
  uint64_t* op_empty = bars + 10;  // [2] MMAs reading the operand set completed
  uint64_t* acc_full = bars + 12;  // [2] accumulator holds a finished item
  uint64_t* acc_empty = bars + 14; // [2] accumulator drained by the epilogue warps
  uint64_t* drain = bars + 16;     // abort path: every issued MMA completed
  uint32_t* tslot = reinterpret_cast<uint32_t*>(smem_raw + L.slot_off);
  const int nitems = p.n_items;
  const uint32_t box_bytes = (uint32_t)(kTcRows * B * sizeof(float));

  if (tid == 0) {
    s_abort = 0;
    for (int q = 0; q < NF; ++q) {
      mbar_init(&fp_full[q], 1);
      mbar_init(&fp_empty[q], kTcConv / 32);
    }
    for (int q = 0; q < 2; ++q) {
      mbar_init(&op_full[q], kTcConv / 32);
      mbar_init(&op_empty[q], 1);
      mbar_init(&acc_full[q], 1);
      mbar_init(&acc_empty[q], 4);
    }
    mbar_init(drain, 1);
    mbar_fence_init();
  }
  if (warp == 0) {
    tmem_alloc(tslot, kTmemCols);
    tmem_relinquish();
  }
  // both operand sets zeroed: the pad columns after L and the groups of
  // H and L past the last band group and the augmentation are never
  // written again
  for (size_t i = tid; i < 2 * L.opb / 16; i += kTcThreads)
    reinterpret_cast<uint4*>(ops)[i] = make_uint4(0u, 0u, 0u, 0u);
  fence_proxy_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;

  // every role walks the same items and stages; an item of a line whose
  // iterations are done (literal schedule) has no stages
  auto item_geom = [&](int w, StatItem& it, int& nst) {
    it = stat_item(p, w);
    nst = (it.r_end - it.r_beg + kTcRows - 1) / kTcRows;
    if (mode == STAT_LITERAL && pass > p.lines[it.line].n_iter) nst = 0;
  };
  bool failed = false;
  int issued[kMaxFpStages] = {0, 0, 0};  // producer: copies per float32 stage

  if (warp == 8) {
    // ---------------- producer
    if (lane == 0) {
      prefetch_tmap(&map);
      int fb = 0;         // float32 stage of the g-th copy: g % NF
      uint32_t fph = 0;   // its phase parity: (g / NF) & 1
      for (int w = blockIdx.x; w < nitems && !failed; w += gridDim.x) {
        StatItem it;
        int nst;
        item_geom(w, it, nst);
        for (int s = 0; s < nst; ++s, (++fb == NF ? (fb = 0, fph ^= 1u) : 0u)) {
          if (!mbar_wait(&fp_empty[fb], fph ^ 1u)) {
            failed = true;
            atomicExch(&s_abort, 1);
            break;
          }
          mbar_arrive_expect_tx(&fp_full[fb], box_bytes);
          // evict-first: the moment partials the initial solve reads next
          // stay in L2
          tma_load_3d_hint(stage(fb), &map, p.band_lo, it.c, it.r_beg + s * kTcRows, &fp_full[fb],
                           l2_policy_evict_first());
          ++issued[fb];
        }
      }
    }
  } else if (warp == 9) {
    // ---------------- issuer
    if (lane == 0) {
      const uint32_t idesc = umma_idesc_bf16_mn(kTcM, 2 * NP);
      const uint32_t idesc_ll = umma_idesc_bf16_mn(kTcM, NP);
      const uint32_t ops_s = smem_u32(ops);
      int g = 0;
      for (int w = blockIdx.x; w < nitems && !failed; w += gridDim.x) {
        StatItem it;
        int nst;
        item_geom(w, it, nst);
        for (int s = 0; s < nst; ++s, ++g) {
          const int sb = g & 1;  // operand set and accumulator of this stage
          if (!mbar_wait(&acc_empty[sb], (uint32_t)(((g >> 1) & 1) ^ 1)) ||
              !mbar_wait(&op_full[sb], (uint32_t)((g >> 1) & 1))) {
            failed = true;
            atomicExch(&s_abort, 1);
            break;
          }
          tc_fence_after();
          const uint32_t acc = tmem + (uint32_t)(sb * L.accw);
          const uint32_t os = ops_s + (uint32_t)(sb * L.opb);
#pragma unroll 1
          for (int kk = 0; kk < kTcRows / 16; ++kk) {
            // A = 128 columns from H's (L's) start: H (L), then garbage
            // rows of D; B = [H | L] (L)
            const uint32_t ga = os + (uint32_t)(kk * 2 * L.kstride);
            const uint64_t dh = umma_smem_desc(ga, (uint32_t)L.kstride, 128);
            const uint64_t dl = umma_smem_desc(ga + (uint32_t)L.lo_off, (uint32_t)L.kstride, 128);
            umma_bf16(acc, dh, dh, idesc, kk > 0 ? 1u : 0u);
            umma_bf16(acc, dl, dl, idesc_ll, 1u);
          }
          umma_commit(&op_empty[sb]);
          umma_commit(&acc_full[sb]);
        }
      }
    }
  } else if (warp >= 10) {
    // ---------------- epilogue: stage accumulator -> running sum -> moments
    // Each stage's D (128 pixels, 16 MMAs) is added in float32 into the
    // item's running sum Q, kept in tensor memory: short accumulation
    // chains on the tensor cores, one rounded add per stage here.
    const int quad = warp & 3;            // a warp may access TMEM lanes 32 (warp % 4) ..
    const int m = quad * 32 + lane;       // row of G
    const int K1E = k1_entries(BA);
    const uint32_t lanes = (uint32_t)(quad * 32) << 16;
    const uint32_t qsum = tmem + lanes + (uint32_t)(2 * L.accw);
    int g = 0;
    for (int w = blockIdx.x; w < nitems && !failed; w += gridDim.x) {
      StatItem it;
      int nst;
      item_geom(w, it, nst);
      // the item's Q, BA x BA column-major (Q_mj at j BA + m): a warp's
      // store of one column is 32 consecutive floats; the reduction forms
      // G = Q + Q^T
      float* dst = reinterpret_cast<float*>(p.k1part + (size_t)it.unit * K1E);
      for (int s = 0; s < nst; ++s, ++g) {
        const int sb = g & 1;
        // warp-uniform decision: tcgen05.ld below needs every lane
        if (!__all_sync(0xffffffffu, mbar_wait(&acc_full[sb], (uint32_t)((g >> 1) & 1)))) {
          failed = true;
          atomicExch(&s_abort, 1);
          break;
        }
        tc_fence_after();
        const uint32_t acc = tmem + lanes + (uint32_t)(sb * L.accw);
        const bool last = s == nst - 1;
        // batches of 32 columns (16-column loads of H^T H + L^T L, H^T L
        // and the running sum, one wait per batch)
        for (int c0 = 0; c0 < NP; c0 += 32) {
          const bool two = c0 + 16 < NP;
          uint32_t hh[32], hl[32], qs[32];
          tmem_ld16(acc + (uint32_t)c0, hh);
          tmem_ld16(acc + (uint32_t)(NP + c0), hl);
          if (s > 0) tmem_ld16(qsum + (uint32_t)c0, qs);
          if (two) {
            tmem_ld16(acc + (uint32_t)(c0 + 16), hh + 16);
            tmem_ld16(acc + (uint32_t)(NP + c0 + 16), hl + 16);
            if (s > 0) tmem_ld16(qsum + (uint32_t)(c0 + 16), qs + 16);
          }
          tmem_wait_ld();
          tmem_regs_after_wait<32>(hh);
          tmem_regs_after_wait<32>(hl);
          if (s > 0) tmem_regs_after_wait<32>(qs);
          // Q = (H^T H + L^T L) / 2 + H^T L  (+ the running sum)
          float q[32];
#pragma unroll
          for (int k = 0; k < 32; ++k) {
            q[k] = fmaf(0.5f, __uint_as_float(hh[k]), __uint_as_float(hl[k]));
            if (s > 0) q[k] += __uint_as_float(qs[k]);
          }
          if (!last) {
            tmem_st16(qsum + (uint32_t)c0, q);
            if (two) tmem_st16(qsum + (uint32_t)(c0 + 16), q + 16);
          } else if (m < BA) {
#pragma unroll
            for (int k = 0; k < 32; ++k) {
              const int j = c0 + k;
              if (j < BA) dst[(size_t)j * BA + m] = q[k];
            }
          }
        }
        if (!last) tmem_wait_st();
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&acc_empty[sb]);
      }
    }
  } else {
    // ---------------- converters (warps 0-7)
    // the reference directions (and in the literal schedule alpha) come from
    // the previous kernels: wait for the last of them.  The producer's copies
    // of the cube, the MMAs and the epilogue need no wait.
    pdl_wait();
    pdl_trigger();
    const LaunchSpan span(p);
    const int e = lane & 1;
    const int slot = warp * 16 + (lane >> 1);  // pixel = K index within a stage
    const bool albedo = (p.flags & MF_ALBEDO) != 0;
    // this lane's byte offset of group f = e + 2 j in an operand set:
    // K group, row within the core matrix, n0 = 4 f -> j * 128 + 8 e
    const size_t kbase = (size_t)(slot >> 3) * L.kstride + (size_t)(slot & 7) * 16 + 8 * e;
    // mask (and alpha) of this lane's pixel, prefetched two stages ahead
    // along the CTA's sequence of (item, stage): a cursor (pw, ps) walks that
    // sequence and a two-deep queue holds what it loaded
    int pw = blockIdx.x, ps = 0, pnst = 0;
    StatItem pit{};
    auto seek = [&]() {  // the first item from pw on with stages
      for (; pw < nitems; pw += gridDim.x) {
        item_geom(pw, pit, pnst);
        if (pnst > 0) return;
      }
    };
    auto fetch = [&](int& m_out, float& a_out) {
      m_out = 0;
      a_out = 0.f;
      if (pw >= nitems) return;
      const int row = pit.r_beg + ps * kTcRows + slot;
      if (row < pit.r_end) {
        const size_t pix = (size_t)row * p.cols + pit.c;
        if (p.mask) m_out = p.mask[pix];
        if (mode == STAT_LITERAL) a_out = p.alpha[pix];
      }
      if (++ps >= pnst) {
        ps = 0;
        pw += gridDim.x;
        seek();
      }
    };
    seek();
    int m_q0, m_q1;
    float a_q0, a_q1;
    fetch(m_q0, a_q0);
    fetch(m_q1, a_q1);
    int g = 0, t = 0;
    int fb = 0;         // float32 stage of the g-th stage: g % NF
    uint32_t fph = 0;   // its phase parity: (g / NF) & 1
    // reference direction of an item's partition, double-buffered by item:
    // the next item's is loaded into registers during the current item and
    // published by the named barrier that ends it
    const float* refsrc = (mode == STAT_INIT ? p.pilot : p.mu0f);
    // ... and its 1 / (m . m) (the pilot's, or the plan's for mu^0), in the
    // slot after the B entries
    auto ref_of = [&](int w) -> float {
      if (w >= nitems || tid > B) return 0.f;
      const StatItem iw = stat_item(p, w);
      const int pw_ = part_of(p, iw.line, iw.c);
      if (tid < B) return refsrc[(size_t)pw_ * B + tid];
      return mode == STAT_INIT ? p.pilot_s[pw_] : p.pscal[(size_t)pw_ * PS_N + PS_INVMU2];
    };
    if (tid <= B) s_ref[tid] = ref_of(blockIdx.x);
    conv_bar();
    // every converter warp walks every item (and reaches every named barrier)
    // even after a failed wait; it only skips the work
    for (int w = blockIdx.x; w < nitems; w += gridDim.x, ++t) {
      StatItem it;
      int nst;
      item_geom(w, it, nst);
      const float* ref = s_ref + (t & 1) * (kMaxB + 4);
      const float ref_next = ref_of(w + gridDim.x);
      const float inv_ref2 = ref[B];
      // the lane's groups of the reference, in registers for the item
      float4 rf[NJ];
#pragma unroll
      for (int j = 0; j < NJ; ++j) {
        const int f = e + 2 * j;
        rf[j] = f < B4 ? reinterpret_cast<const float4*>(ref)[f] : make_float4(0.f, 0.f, 0.f, 0.f);
      }
      for (int s = 0; s < nst; ++s, ++g, (++fb == NF ? (fb = 0, fph ^= 1u) : 0u)) {
        const int m_cur = m_q0;
        const float a_cur = a_q0;
        m_q0 = m_q1;
        a_q0 = a_q1;
        fetch(m_q1, a_q1);
        if (__any_sync(0xffffffffu, failed || *(volatile int*)&s_abort)) {
          failed = true;
          continue;
        }
        const int sb = g & 1;
        const int row = it.r_beg + s * kTcRows + slot;
        const bool inb = row < it.r_end;
        // warp-uniform decision: the shuffles below need every lane
        const bool ok_w = mbar_wait(&fp_full[fb], fph) &&
                          mbar_wait(&op_empty[sb], (uint32_t)(((g >> 1) & 1) ^ 1));
        if (!__all_sync(0xffffffffu, ok_w)) {
          failed = true;
          atomicExch(&s_abort, 1);
          continue;
        }
        unsigned char* H = ops + (size_t)sb * L.opb + kbase;
        unsigned char* Lo = H + L.lo_off;
        const float4* px = reinterpret_cast<const float4*>(stage(fb) + (size_t)slot * B);
        float4 x[NJ];
#pragma unroll
        for (int j = 0; j < NJ; ++j) {
          const int f = e + 2 * j;
          x[j] = (inb && f < B4) ? px[f] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        // every band finite <=> the dot with the (finite) reference is
        // finite (x * 0 is NaN for x = +-Inf or NaN)
        const float dot = pair_dot2<NJ>(x, rf);
        // every lane's x is in registers (the dot consumed it): only now
        // release the float32 stage to the next TMA copy, which must not
        // overtake a pending load
        __syncwarp();
        if (lane == 0) mbar_arrive(&fp_empty[fb]);
        const bool valid = inb && isfinite(dot) && m_cur == 0;
        const float rho = dot * inv_ref2;
        split_residual2<NJ>(x, rf, rho);
        float4 aug = make_float4(0.f, 0.f, 0.f, 0.f);
        if (valid) {
          float bcf = 0.f;
          if (mode == STAT_LITERAL) {
            const float r = albedo ? rho : 1.f;
            bcf = r > 0.f ? -(r * a_cur) : 0.f;
          }
          aug = make_float4(rho - 1.f, bcf, 1.f, 0.f);
        }
        // an excluded pixel contributes nothing (rare: a warp-uniform branch)
        if (__any_sync(0xffffffffu, !valid) && !valid) {
#pragma unroll
          for (int j = 0; j < NJ; ++j) x[j] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        // groups f = e + 2 j of the augmented vector [e, rho - 1, bcf, 1, 0 ..]:
        // the augmentation at f = B4, then the bands (x[j] is zero past B4
        // for a valid pixel, since the reference is) except the group the
        // augmentation took (the same lane's).  Groups that no stage writes
        // were zeroed at kernel start.
        const int j_aug = e == (B4 & 1) ? (B4 >> 1) : -1;
        {
          uint2 hi, lo;
          split_bf16x4(aug, hi, lo);
          if (j_aug >= 0) {
            *reinterpret_cast<uint2*>(H + (size_t)j_aug * 128) = hi;
            *reinterpret_cast<uint2*>(Lo + (size_t)j_aug * 128) = lo;
          }
        }
#pragma unroll
        for (int j = 0; j < NJ; ++j) {
          uint2 hi, lo;
          split_bf16x4(x[j], hi, lo);
          if (j != j_aug && 4 * (e + 2 * j) < NP) {
            *reinterpret_cast<uint2*>(H + (size_t)j * 128) = hi;
            *reinterpret_cast<uint2*>(Lo + (size_t)j * 128) = lo;
          }
        }
        fence_proxy_async_smem();  // operand writes -> tensor core (async proxy)
        __syncwarp();
        if (lane == 0) mbar_arrive(&op_full[sb]);
      }
      if (tid <= B) s_ref[((t + 1) & 1) * (kMaxB + 4) + tid] = ref_next;
      conv_bar();
    }
  }
  if (failed) atomicExch(&s_abort, 1);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (s_abort) {
    // bounded waits for this CTA's copies and MMAs still in flight, then
    // release the tensor memory
    if (warp == 8 && lane == 0)
      for (int q = 0; q < NF; ++q)
        if (issued[q] > 0) mbar_wait(&fp_full[q], (uint32_t)((issued[q] - 1) & 1));
    if (warp == 9 && lane == 0) {
      umma_commit(drain);
      mbar_wait(drain, 0);
    }
    if (tid == 0)
      for (int w = blockIdx.x; w < nitems; w += gridDim.x) {
        const StatItem iw = stat_item(p, w);
        p.status[part_of(p, iw.line, iw.c)] = MF_ERR_TIMEOUT;
      }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
  }
  if (warp == 0) tmem_dealloc(tmem, kTmemCols);
}

#define MF_NJ_CASES(X) X(8) X(9) X(10) X(12)

cudaError_t stats_tc_set_attributes(int nj, size_t smem) {
#define MF_CASE(NJ)                                                                    \
  case NJ:                                                                             \
    return cudaFuncSetAttribute(stats_tc_kernel<NJ>,                                   \
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  switch (nj) { MF_NJ_CASES(MF_CASE) }
#undef MF_CASE
  return cudaErrorInvalidValue;
}

void pilot_launch(cudaStream_t s, const Params& p) {
  pilot_kernel<<<(p.P + 3) / 4, 128, 0, s>>>(p);
}

void stats_tc_launch(int nj, int grid, size_t smem, cudaStream_t s, const CUtensorMap& map,
                     const Params& p, int mode, int pass) {
#define MF_CASE(NJ)                                                             \
  case NJ:                                                                      \
    launch_kernel(stats_tc_kernel<NJ>, grid, kTcThreads, smem, s, p.pdl != 0, map, p, mode, \
                  pass);                                                          \
    return;
  switch (nj) { MF_NJ_CASES(MF_CASE) }
#undef MF_CASE
}

}  // namespace mf
