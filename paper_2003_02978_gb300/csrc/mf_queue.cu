// Persistent form of a retrieval (MF_PERSISTENT): after the statistics
// pass, ONE launch runs the initial solves, every pixel pass and every
// iteration solve of every line of the plan, as work items taken from a
// queue (Fig. 1 per line; Sec. II-E: partitions and flightlines are
// independent problems).
//
// Items.  Per pass k = 0 .. n_iter_max and line l there are two groups: the
// solves of l's partitions, S(k, l) (solve_init_part for k = 0,
// solve_iter_part otherwise), and l's pixel CTAs, X(k, l) (pixel_block).  A
// pass lists its groups as
//   S(k,0) S(k,1) X(k,0) S(k,2) X(k,1) ... S(k,L-1) X(k,L-2) X(k,L-1)
// so a line's solves come one line ahead of its pixel blocks, and every
// item's dependencies are in groups listed before it:
//   X(k, l) tile T   needs S(k, l) of every partition with a column in T;
//   S(k, l) part P   (k >= 1) needs X(k-1, l) of every tile with a column of P.
// CTAs (one wave: SMs x resident CTAs) take items in list order from one
// atomic counter and finish each before taking the next.  The queue cannot
// deadlock whatever the number of resident CTAs: the earliest unfinished item
// has all its dependencies finished (they are earlier) and is held by a
// running CTA.  A line whose N_iter is below k skips its items of pass k
// without signalling them (nothing waits for them, and a skipped solve's
// signal could overtake the partition's previous solve).
//
// Completion.  S items store k + 1 into the partition's progress word, X
// items add 1 to the tile's counter (which reaches (k + 1) n_rb once pass k
// of the tile is done): after a barrier over the item's writes one thread
// fences and releases.  Waits load with acquire semantics, then a barrier:
// what the producer wrote is visible to every thread of the consumer,
// including the L^-1 that the iteration solve then copies by the async
// proxy (proxy fence before the copy).  Every wait is bounded (Params::q_wait_ns) and also ends when
// another CTA has raised the abort word; a CTA whose wait or copy runs out
// raises it and leaves, and the host reports MF_ERR_TIMEOUT.
//
// The arithmetic of each item is that of the per-pass kernels (the same
// device functions, the same fixed summation orders), so the result is
// bit-identical to the launch-per-pass sequence.
#include "mf_pixel_body.cuh"
#include "mf_solve_body.cuh"

namespace mf {

namespace {

static_assert(kPixThreads == kThreads, "the work-queue kernel runs pixel and solve items");

__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ int ld_relaxed(const int* p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(int* p, int v) {
  asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void red_release_add(int* p, int v) {
  asm volatile("red.release.gpu.global.add.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// the words of Params::q_words
struct Queue {
  unsigned long long* head;  // next item
  int* abort;                // raised by a CTA whose wait ran out
  int* solve_done;           // (P) passes whose solve completed
  int* pix_done;             // (n_lines n_ct) pixel items completed, all passes
};
__device__ __forceinline__ Queue queue_of(const Params& p) {
  int* w = p.q_words;
  return {reinterpret_cast<unsigned long long*>(w), w + 2, w + kQueueHead,
          w + kQueueHead + p.P};
}

// Every thread of the CTA: wait until flags[i] >= target for all i < n
// (thread t takes i = t, t + kThreads, ...).  False (for the whole CTA)
// when a wait ran out, which raises the abort word, or saw it raised.
__device__ bool wait_all_geq(const Params& p, const Queue& q, const int* flags, int n,
                             int target) {
  bool ok = true;
  for (int i = threadIdx.x; i < n && ok; i += kThreads) {
    const int* f = flags + i;
    if (ld_acquire(f) >= target) continue;
    const unsigned long long t0 = globaltimer_ns();
    unsigned ns = 32;
    while (ld_acquire(f) < target) {
      if (ld_relaxed(q.abort) != 0) {
        ok = false;
        break;
      }
      if (globaltimer_ns() - t0 > (unsigned long long)p.q_wait_ns) {
        atomicExch(q.abort, 1);
        ok = false;
        break;
      }
      __nanosleep(ns);
      if (ns < 256) ns *= 2;
    }
  }
  // the acquiring loads, then the barrier: every thread's later reads see
  // what the producers wrote before their release
  return __syncthreads_and(ok) != 0;
}

// the item's writes by every thread, the barrier, then one fenced release
__device__ __forceinline__ void signal_store(int* f, int v) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    st_release(f, v);
  }
}
__device__ __forceinline__ void signal_add(int* f) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    red_release_add(f, 1);
  }
}

enum : int { Q_SOLVE = 0, Q_PIXEL = 1 };
struct QItem {
  int pass, kind, line, index;  // index: partition, or pixel CTA (as numbered by the plan)
};
__device__ __forceinline__ QItem queue_item(const Params& p, unsigned long long item) {
  const int L = p.n_lines;
  const unsigned long long per_pass = (unsigned long long)p.q_groups[2 * L];
  QItem it;
  it.pass = (int)(item / per_pass);
  const int r = (int)(item - (unsigned long long)it.pass * per_pass);
  int lo = 0, hi = 2 * L - 1;  // the group: last q_groups[g] <= r
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (p.q_groups[mid] <= r) lo = mid;
    else hi = mid - 1;
  }
  const int g = lo, off = r - p.q_groups[g];
  if (g == 0) {
    it.kind = Q_SOLVE;
    it.line = 0;
  } else if (g == 2 * L - 1) {
    it.kind = Q_PIXEL;
    it.line = L - 1;
  } else if (g & 1) {
    it.kind = Q_SOLVE;
    it.line = (g + 1) / 2;
  } else {
    it.kind = Q_PIXEL;
    it.line = g / 2 - 1;
  }
  it.index = it.kind == Q_SOLVE ? it.line * p.Pl + off : p.lines[it.line].blk0 + off;
  return it;
}

// the next item into *slot (one thread)
__device__ __forceinline__ void take_next(const Params& p, unsigned long long* slot) {
  const Queue q = queue_of(p);
  *slot = ld_relaxed(q.abort) != 0 ? ~0ull : atomicAdd(q.head, 1ull);
}

// A solve item: the dependency wait, the solve and its signal.  The solves
// and the queue's helpers run out of line with their own register
// allocation, so that the pixel stream inlined into the kernel is compiled
// about as in the per-pass kernel, its parameters read from the constant
// bank (measured: all inlined, the kernel spilled 248 bytes and a pixel
// item took 146 us against the per-pass kernel's 108 us; in this form 116
// bytes and 108 us).
__device__ __noinline__ bool queue_solve(const Params& p, const QItem it,
                                         unsigned char* smem_raw, uint64_t* xbar,
                                         uint32_t& ph_x) {
  const Queue q = queue_of(p);
  const int part = it.index;
  bool ok = true;
  if (it.pass == 0) {
    solve_init_part<true>(p, part, smem_raw);
  } else {
    ok = solve_iter_part<true>(p, SOLVE_FUSED, it.pass, part, smem_raw, xbar, ph_x, [&] {
      // pass - 1 of the tiles over the partition's columns
      const int c0 = part_col0(p, part), c1 = c0 + part_ncols(p, part) - 1;
      const int t0 = c0 / kTileCols;
      return wait_all_geq(p, q, q.pix_done + it.line * p.n_ct + t0, c1 / kTileCols - t0 + 1,
                          it.pass * p.lines[it.line].n_rb);
    });
  }
  if (ok) signal_store(q.solve_done + part, it.pass + 1);
  return ok;
}

// a pixel item's dependency wait: this pass's solves of the tile's partitions
__device__ __noinline__ bool pixel_ready(const Params& p, const QItem it) {
  const int ct = (it.index - p.lines[it.line].blk0) % p.n_ct;
  const int c0t = ct * kTileCols;
  const int c1 = min(c0t + kTileCols, p.cols) - 1;
  const int first = part_of(p, it.line, c0t);
  const Queue q = queue_of(p);
  return wait_all_geq(p, q, q.solve_done + first, part_of(p, it.line, c1) - first + 1,
                      it.pass + 1);
}

template <int NJ>
__global__ void __launch_bounds__(kThreads, pix_ctas_per_sm(NJ))
    queue_kernel(const __grid_constant__ CUtensorMap map, const __grid_constant__ Params p,
                 int n_iter_max) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bars[kPixBars + 1];  // pixel items', the L^-1 copy's
  // the CTA's queue state lives in shared memory (or is recomputed from the
  // constant bank), not in registers across the pixel stream
  __shared__ PixPhases s_ph;
  __shared__ unsigned long long s_item;
  const LaunchSpan span(p);
  const int tid = threadIdx.x;
  if (tid == 0) {
    pixel_bars_init(bars);
    mbar_init(&bars[kPixBars], 1);
    mbar_fence_init();
    s_ph = PixPhases{};
  }
  uint32_t ph_x = 0;
  for (;;) {
    __syncthreads();
    if (tid == 0) {
      // the last item's generic shared-memory writes before this item's
      // copies into the same bytes
      fence_proxy_async_smem();
      take_next(p, &s_item);
    }
    __syncthreads();
    const unsigned long long item = s_item;
    __syncthreads();  // s_item is rewritten only once every thread has read it
    if (item >= (unsigned long long)(n_iter_max + 1) * (unsigned long long)p.q_groups[2 * p.n_lines])
      break;  // past the end, or the queue stopped
    const QItem it = queue_item(p, item);
    if (it.pass > p.lines[it.line].n_iter) continue;  // past the line's N_iter: nothing to do
    bool ok = true;
    if (it.kind == Q_SOLVE) {
      ok = queue_solve(p, it, smem_raw, &bars[kPixBars], ph_x);
    } else {
      ok = pixel_block<NJ, true>(map, p, it.pass == 0 ? PIX_INIT : PIX_ITER,
                                 it.pass < n_iter_max, it.pass, it.index, smem_raw, bars, s_ph,
                                 [&] { return pixel_ready(p, it); });
      if (ok) {
        // this item again from its index, not kept live across the stream
        const QItem jt = queue_item(p, item);
        const int ct = (jt.index - p.lines[jt.line].blk0) % p.n_ct;
        signal_add(queue_of(p).pix_done + jt.line * p.n_ct + ct);
      }
    }
    if (!ok) {
      if (tid == 0) atomicExch(queue_of(p).abort, 1);
      break;
    }
  }
}

}  // namespace

#define MF_NJ_CASES(X) X(1) X(2) X(4) X(6) X(8) X(9) X(10) X(12) X(16)

cudaError_t queue_set_attributes(int nj, size_t smem) {
#define MF_CASE(NJ)                                                                   \
  case NJ:                                                                            \
    return cudaFuncSetAttribute(queue_kernel<NJ>,                                     \
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  switch (nj) { MF_NJ_CASES(MF_CASE) }
#undef MF_CASE
  return cudaErrorInvalidValue;
}

int queue_ctas_per_sm(int nj, size_t smem) {
  int n = 0;
#define MF_CASE(NJ)                                                                        \
  case NJ:                                                                                 \
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, queue_kernel<NJ>, kThreads, smem) \
        != cudaSuccess)                                                                    \
      return 0;                                                                            \
    return n;
  switch (nj) { MF_NJ_CASES(MF_CASE) }
#undef MF_CASE
  return 0;
}

void queue_launch(int nj, int grid, size_t smem, cudaStream_t s, const CUtensorMap& map,
                  const Params& p, int n_iter_max) {
#define MF_CASE(NJ)                                                                       \
  case NJ:                                                                                \
    launch_kernel(queue_kernel<NJ>, grid, kThreads, smem, s, false, map, p, n_iter_max); \
    return;
  switch (nj) { MF_NJ_CASES(MF_CASE) }
#undef MF_CASE
}

}  // namespace mf
