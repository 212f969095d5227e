/*
 * mf.h -- C ABI of the GB300-native sparse, albedo-corrected matched filter.
 *
 * Method: Foote et al., "Fast and Accurate Retrieval of Methane Concentration
 * from Imaging Spectrometer Data Using Sparsity Prior", IEEE TGRS 2020
 * (arXiv 2003.02978).  For each detector partition of a radiance cube the
 * library runs the procedure of Fig. 1 (Algorithm AlbedoReWeightL1Filter):
 * background mean and covariance, albedo factor r_i (Eq. (7)), target
 * t = mu (.) s (Eq. (9)), the matched-filter initial estimate (Eq. (3)
 * divided by r_i), then N_iter reweighted-l1 iterations: weights
 * w_i = 1/(alpha_i + eps) (Eq. (5)), mean and covariance re-estimated with the
 * current enhancement removed (Eqs. (10)-(11)), and the non-negative
 * shrinkage update of alpha_i (Eq. (6) with the albedo factor of Sec. II-C).
 *
 * Conventions shared by every entry point:
 *  - Cube layout is BIP: cube[(row * cols + col) * bands_total + band], float32,
 *    C-contiguous.  The band window is [band_lo, band_hi); B = band_hi - band_lo.
 *  - A partition (Sec. II-E) is a group of col_group adjacent columns; the
 *    remaining columns form one last smaller group.  P = ceil(cols / col_group).
 *  - Device pointers are CUDA device (or managed) memory owned by the caller.
 *    "stream" is a cudaStream_t passed as void* (NULL = legacy default stream).
 *  - Functions return mf_status.  Argument/shape errors are returned
 *    synchronously and nothing is enqueued.  Per-partition numerical failures
 *    (covariance not positive definite, N <= B) are recorded on the device and
 *    read back with mf_plan_status(); such a partition gets alpha = NaN on its
 *    valid pixels.  Masked or non-finite pixels get alpha = 0 and are excluded
 *    from every statistic.
 *  - mf_retrieve allocates nothing and never synchronises; a plan may be used
 *    by one stream at a time.
 */
#ifndef MF_H_
#define MF_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mf_plan_s* mf_plan_t;

typedef enum {
  MF_OK = 0,
  MF_ERR_INVALID_ARG = 1,      /* bad pointer, size, window, flag combination */
  MF_ERR_CUDA = 2,             /* a CUDA runtime call failed (see mf_last_error) */
  MF_ERR_OOM = 3,              /* workspace allocation failed in mf_plan */
  MF_ERR_NOT_SPD = 4,          /* per partition: covariance not positive definite */
  MF_ERR_NONFINITE_INPUT = 5,  /* k, lambda or eps not finite */
  MF_ERR_TIMEOUT = 6,          /* a bounded device-side wait expired */
  MF_ERR_INTERNAL = 7,
  MF_ERR_UNSUPPORTED = 8       /* shape outside what this build supports */
} mf_status;

enum { MF_BIP = 0 };                       /* layout */
/* precision of the covariance accumulation:
 *   MF_FP32       float32 products, double-float partial sums (SIMT)
 *   MF_BF16SPLIT  every augmented pixel split into bf16 hi + lo and the
 *                 moments H^T H + H^T L + L^T H accumulated in float32 on
 *                 the tensor cores; supported for 64 <= B <= 92 */
enum { MF_FP32 = 0, MF_BF16SPLIT = 1 };

/* flags */
#define MF_ALBEDO            1u  /* albedo factor r_i of Eq. (7); off: r_i = 1 (Fig. 1 caption) */
#define MF_SPARSE            2u  /* reweighted-l1 weights of Eq. (5); off: w = 0 (Fig. 1 caption) */
#define MF_LITERAL           4u  /* re-accumulate C^k by a full pass and refactor it every
                                    iteration, as Fig. 1 prints it; off: exact rank-3 update of
                                    C^0 (same result up to rounding) */
#define MF_PENALTY_NO_ALBEDO 8u  /* penalty lambda*w_i/r_i instead of lambda*w_i */
#define MF_PERSISTENT       16u  /* after the statistics pass, one persistent launch runs the
                                    initial solves, every pixel pass and every iteration solve
                                    of every line as work items of a dependency-ordered queue
                                    (same results, bit for bit, as the launch-per-pass
                                    sequence); not with MF_LITERAL.  Each dependency wait is
                                    bounded (MF_QUEUE_WAIT_MS, default 2000): one that runs out
                                    stops the queue and every partition's status reads
                                    MF_ERR_TIMEOUT */

typedef struct {
  int64_t rows;         /* along-track lines */
  int64_t cols;         /* cross-track detectors */
  int64_t bands_total;  /* bands stored per pixel */
  int32_t band_lo;      /* first band of the window */
  int32_t band_hi;      /* one past the last band of the window */
  int32_t col_group;    /* adjacent detectors per partition (>= 1) */
  int32_t layout;       /* MF_BIP */
  int32_t precision;    /* MF_FP32 | MF_BF16SPLIT */
  uint32_t flags;       /* MF_ALBEDO | MF_SPARSE | MF_LITERAL | MF_PENALTY_NO_ALBEDO |
                           MF_PERSISTENT */
} mf_desc;

/* Validate the descriptor and allocate every device buffer a retrieval of
 * this shape needs, once (statistics, Cholesky factors, per-block partial
 * sums, counters, status).  Supported: 8 <= B <= 128, B % 4 == 0,
 * band_lo % 4 == 0, bands_total % 4 == 0 (16-byte aligned pixel windows),
 * rows * col_group > B.  Uses the current CUDA device.  *out is owned by the
 * caller and released with mf_destroy.
 * Environment read here (all optional): MF_GRAPH=0 launches the kernels
 * directly instead of replaying a CUDA graph; MF_RB_ROWS / MF_SC_ROWS set the
 * rows per pixel-kernel CTA / per statistics item (as mf_tuning); MF_PDL=0
 * launches every kernel in plain stream order (default: programmatic
 * dependent launch for the statistics and solve kernels); MF_PF_STAGES (default
 * 4, 0 = off) sets how many stages of every pixel-kernel CTA the solve
 * kernels prefetch into L2 for the pass that follows them;
 * MF_FORCE_DIRECT=1 (a test hook) sends every fused iteration's solve through
 * the direct factorisation of C^k that otherwise serves only ill-conditioned
 * Woodbury systems.  MF_FAULT (a fault-injection hook for tests; nothing in
 * it faults the GPU) forces a failure path: "alloc" makes mf_plan return
 * MF_ERR_OOM before any CUDA call; "notspd" reports every partition's
 * initial covariance as not positive definite (MF_ERR_NOT_SPD, alpha NaN);
 * "timeout" makes every pixel-kernel CTA of the first pass wait 2000 cycles
 * on a barrier nothing arrives on, so that it records MF_ERR_TIMEOUT (after
 * its own copies have landed) and the later passes write NaN. */
mf_status mf_plan(const mf_desc* desc, mf_plan_t* out);

/* Release a plan and its device memory (synchronises the device first). */
void mf_destroy(mf_plan_t plan);

/* Number of partitions P of the plan. */
int64_t mf_num_partitions(mf_plan_t plan);

/* One full retrieval, Fig. 1 (Algorithm AlbedoReWeightL1Filter), on every
 * partition, enqueued on `stream`.
 *   cube       device, (rows, cols, bands_total) float32 BIP
 *   k          device, B float32: unit absorption spectrum s of Sec. II-D
 *   lambda     multiplier on the paper's weight w_i (1 = Fig. 1 verbatim,
 *              0 = no sparsity); eps the constant of Eq. (5), > 0
 *   n_iter     reweighting iterations N_iter >= 0; with 0 the initial
 *              estimate alpha^0 is returned unclamped (Table I, non-iterative rows)
 *   mask       device (rows, cols) uint8, nonzero = excluded, or NULL
 *   alpha_init device (rows, cols) float32 replacing alpha^0, or NULL
 *   alpha_out  device (rows, cols) float32: alpha^{N_iter} in ppm*m
 *   albedo_out device (rows, cols) float32: r_i (1 when MF_ALBEDO is off;
 *              0 on masked pixels), or NULL
 * Allocates nothing, does not synchronise. */
mf_status mf_retrieve(mf_plan_t plan, const float* cube, const float* k, double lambda,
                      double eps, int32_t n_iter, const uint8_t* mask,
                      const float* alpha_init, float* alpha_out, float* albedo_out,
                      void* stream);

/* mf_retrieve with HOST buffers (pageable or pinned).  Copies the cube, k
 * and mask to plan-owned device staging (allocated on the first call and
 * reused), retrieves, copies alpha back and synchronises `stream` before
 * returning.  Same arguments as mf_retrieve, all host pointers. */
mf_status mf_retrieve_host(mf_plan_t plan, const float* cube, const float* k, double lambda,
                           double eps, int32_t n_iter, const uint8_t* mask,
                           float* alpha_out, void* stream);

/* mf_retrieve_host for a stream of cubes: the same arguments (HOST
 * pointers; cube, mask and alpha_out in pinned memory for the copies to be
 * asynchronous), but the call returns without synchronising, so that the
 * copy of the next call's cube overlaps this call's retrieval.  Two sets of
 * plan-owned device staging (allocated on the first call, 2 x (cube + mask
 * + alpha) bytes) alternate between calls, with a plan-owned copy stream:
 * call n copies its inputs in on that stream once call n - 2's retrieval
 * and output copy are done, the retrieval and the copy of alpha out run on
 * `stream` after the inputs have landed.  alpha_out holds the result once
 * `stream` has been synchronised after the call; the host buffers must stay
 * alive and unchanged until then.  Errors as mf_retrieve_host. */
mf_status mf_retrieve_host_async(mf_plan_t plan, const float* cube, const float* k, double lambda,
                                 double eps, int32_t n_iter, const uint8_t* mask,
                                 float* alpha_out, void* stream);

/* mf_retrieve (no alpha_init, no albedo output) that also writes the
 * objective of every iterate, the energy whose decrease Fig. 5 tracks (Sec.
 * III-B): for iterate k = 0..n_iter of partition j,
 *   energy_out[j * (n_iter + 1) + k] = sum_i f_i(alpha_i^k),
 *   f_i(a) = d^T (C^k)^-1 d + 2 pen_i r_i a,  d = (L_i - mu^k) - r_i a t^k,
 * over the partition's valid pixels: the bracket of Eq. (8) in the form the
 * shrinkage step of Fig. 1 minimises exactly (pen_i = lambda w_i^k, 0 at
 * k = 0; alpha^0 is the unclamped initial estimate), with mu^k, C^k, t^k of
 * iterate k.  The quadratic term is summed in closed form per partition,
 * N tr((C^k)^-1 S^k) with S^k the scatter of the pixels about mu^k.
 *   energy_out  device, (P, n_iter + 1) float64, 8-byte aligned; NaN for a
 *               partition that fails, and for an iterate whose covariance
 *               took the direct (non-Woodbury) factorisation
 * Single-line plans, fused schedule (MF_LITERAL: MF_ERR_UNSUPPORTED).  Runs
 * the kernels directly (no graph).  Allocates nothing, does not synchronise. */
mf_status mf_retrieve_energy(mf_plan_t plan, const float* cube, const float* k, double lambda,
                             double eps, int32_t n_iter, const uint8_t* mask, float* alpha_out,
                             double* energy_out, void* stream);

/* Batched form: many flightlines of uneven length in one retrieval.  The
 * lines are stacked along rows in one BIP cube: line l is rows
 * [line_rows[0] + ... + line_rows[l-1], ... + line_rows[l]) and desc->rows is
 * the sum; cols, the band window, col_group, precision and flags are shared.
 * Every line has its own partitions (Sec. II-E), P = n_lines x
 * ceil(cols / col_group) in all, line-major, and its own statistics, lambda
 * and iteration count; every kernel of the retrieval covers all lines at once
 * (a line whose iterations are done skips the later passes).  Errors as
 * mf_plan; line_rows (host, n_lines) must be positive. */
mf_status mf_plan_batched(const mf_desc* desc, const int64_t* line_rows, int32_t n_lines,
                          mf_plan_t* out);

/* Launch-shape choices of a plan (0 = the library's default, which sizes the
 * grids from the SM count):
 *   pixel_rows  rows per pixel-kernel CTA (rounded up to 8; per line, the
 *               line is split evenly into blocks of at most this many rows)
 *   stat_rows   rows per statistics work item (rounded up to 128; the
 *               BF16-split form accepts at most 1024 before its stated bound
 *               is untested)
 *   use_graph   < 0: launch the kernels directly instead of replaying a CUDA
 *               graph of the retrieval */
typedef struct {
  int32_t pixel_rows;
  int32_t stat_rows;
  int32_t use_graph;
} mf_tuning;

/* mf_plan / mf_plan_batched with launch-shape choices (an autotuner's
 * output); line_rows NULL means one line of desc->rows.  tuning may be
 * NULL. */
mf_status mf_plan_ex(const mf_desc* desc, const int64_t* line_rows, int32_t n_lines,
                     const mf_tuning* tuning, mf_plan_t* out);

/* Number of lines of a plan (1 for mf_plan), or -1 for a null plan. */
int32_t mf_num_lines(mf_plan_t plan);

/* One retrieval of every line of a batched plan, enqueued on `stream`
 * (Fig. 1 per line).  cube, mask, alpha_out: device, stacked as the plan's
 * lines (rows = sum of line rows); k: device, B float32, shared; lambda and
 * n_iter: HOST arrays of n_lines (copied before return; lambda >= 0 finite,
 * 0 <= n_iter <= 100000); eps > 0 shared.  No alpha_init or albedo output.
 * Allocates nothing; does not synchronise unless lambda or n_iter changed
 * since the previous call (it then waits for that call's table upload). */
mf_status mf_retrieve_batched(mf_plan_t plan, const float* cube, const float* k,
                              const double* lambda, double eps, const int32_t* n_iter,
                              const uint8_t* mask, float* alpha_out, void* stream);

/* Differentiation form: a retrieval checkpointed for the backward pass.
 *
 * mf_ckpt_bytes: device bytes of a checkpoint for n_iter iterations (alpha^k
 * of every pass, per partition and pass mu^k, t^k, v^k, g^k, q^k and the
 * moments of beta, plus every buffer the backward pass needs; with cube_grad
 * also two coefficients per pixel and pass for the cube gradient).  0 for a
 * null plan.
 *
 * mf_retrieve_train: mf_retrieve (no alpha_init, no albedo output) that also
 * writes the checkpoint to `ckpt` (device, caller-owned, 256-byte aligned,
 * mf_ckpt_bytes long).  Single-line plans of the fused schedule only (no
 * MF_LITERAL; the literal schedule computes the same C^k); otherwise
 * MF_ERR_UNSUPPORTED.  The cube, k and mask must stay unchanged until the
 * backward pass.
 *
 * mf_retrieve_backward: the adjoint of that retrieval (the unrolled
 * iterations of Fig. 1 reversed, see mf_backward.cu) for the output adjoint
 * grad_alpha (device, rows x cols): grad_k (device, B float32, gradient with
 * respect to the unit absorption spectrum s), grad_lambda (device, 1
 * float32), grad_cube (device, rows x cols x B float32 over the band
 * window, or NULL; needs cube_grad at the forward).  Masked and non-finite
 * pixels and partitions that failed get zero gradient.  The clamp max(., 0)
 * has subgradient 0 at the kink.  Enqueued on `stream`; allocates nothing. */
size_t mf_ckpt_bytes(mf_plan_t plan, int32_t n_iter, int32_t cube_grad);
mf_status mf_retrieve_train(mf_plan_t plan, const float* cube, const float* k, double lambda,
                            double eps, int32_t n_iter, const uint8_t* mask, float* alpha_out,
                            void* ckpt, int32_t cube_grad, void* stream);
mf_status mf_retrieve_backward(mf_plan_t plan, const void* ckpt, const float* grad_alpha,
                               float* grad_k, float* grad_lambda, float* grad_cube,
                               void* stream);

/* Background statistics of the last retrieval's initialisation (Fig. 1,
 * initial mean and covariance): mu0 (P, B) and cov0 (P, B, B), float64
 * DEVICE buffers.  Ordered after the retrieval on `stream`; synchronises it
 * (diagnostic read-back, not for the hot path). */
mf_status mf_background(mf_plan_t plan, double* mu0, double* cov0, void* stream);

/* Copy the per-partition status of the last retrieval to `status` (HOST,
 * P int32, values of mf_status).  Synchronises the plan's last stream.
 * Returns MF_OK if every partition succeeded, else the first failure. */
mf_status mf_plan_status(mf_plan_t plan, int32_t* status);

/* Kernel timing for roofline reporting.  While enabled, every kernel the
 * plan launches is bracketed by two CUDA events on its stream (a few
 * microseconds of host overhead per launch, none on the device). */
mf_status mf_profile(mf_plan_t plan, int32_t enable);

/* Read and reset the timings accumulated since the last read: for kind i
 * (0 = statistics kernel, 1 = pixel kernel, 2 = solve kernels), ms[i] is the
 * summed device time
 * and launches[i] the number of launches; n_kinds entries are written (HOST
 * arrays).  Synchronises the plan's last stream. */
mf_status mf_profile_read(mf_plan_t plan, double* ms, int64_t* launches, int32_t n_kinds);

/* Device timeline for roofline reporting of the retrieval as it runs (one
 * CUDA graph, no events between kernels).  While enabled, thread 0 of every
 * CTA of every kernel a retrieval launches records the GPU's global timer at
 * its start and exit into a slot of that launch (two 64-bit atomics per CTA);
 * the first enable allocates the 64 KB slot buffer (MF_ERR_OOM if it cannot).
 * Enabling or disabling re-captures the plan's graph on the next call. */
mf_status mf_timeline(mf_plan_t plan, int32_t enable);

/* Read and clear the timeline of the last retrieval (call it after every
 * retrieval to be measured).  For launch i < *n (in launch order, at most
 * cap): start_us[i] / end_us[i] are its first CTA's start and last CTA's end
 * in microseconds after the retrieval's earliest start (-1 for a launch that
 * ran no CTA), kind[i] its kernel kind as in mf_profile_read (HOST arrays of
 * cap entries).  Synchronises the device. */
mf_status mf_timeline_read(mf_plan_t plan, double* start_us, double* end_us, int32_t* kind,
                           int32_t cap, int32_t* n);

/* Initial background statistics of every partition -- the mean mu^0 and
 * covariance C^0 of Fig. 1's initialisation, as mf_background returns them
 * after a retrieval -- without allocating any device memory.  The paper has
 * no counterpart: this exists for callers that may not allocate device memory
 * once running (real-time processing that forbids allocation after start-up,
 * hosts whose device memory belongs to another allocator that this library
 * cannot call), which therefore cannot create a plan.
 *   desc   shape, band window and col_group (flags and precision unused)
 *   cube   device (rows, cols, bands_total) float32 BIP, 16-byte aligned
 *   mask   device (rows, cols) uint8, nonzero = excluded, or NULL
 *   mu0    device (P, B) float64 output;  cov0 device (P, B, B) float64 output
 *          (NaN for a partition with N <= B valid pixels)
 * The per-block partial moments live in a fixed 64 MiB file-scope device
 * array that every GPU loading the library holds until exit; shapes whose
 * moments do not fit (P * col_group * 8 * K bytes, K = 16 * nb (nb + 1) / 2,
 * nb = (B + 12) / 4: the bands, eight direction coefficients, the target
 * coefficient and the constant, rounded up; about 30 KB per detector column
 * at B = 72) return
 * MF_ERR_UNSUPPORTED and enqueue nothing.  The first call on each device
 * looks up the array's device address (cudaGetSymbolAddress) and sets kernel
 * attributes: make it before any stream capture; after a cudaDeviceReset the
 * cached address is stale and the entry point must not be called again.
 * Calls share the array (each rewrites its line table and clears its status
 * words): calls that overlap on the GPU race.  Enqueued on `stream`, no
 * synchronisation. */
mf_status mf_background_noalloc(const mf_desc* desc, const float* cube, const uint8_t* mask,
                                double* mu0, double* cov0, void* stream);

/* Static description of a status code. */
const char* mf_status_string(mf_status s);

/* Message of the last error raised on the calling thread ("" if none). */
const char* mf_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* MF_H_ */
