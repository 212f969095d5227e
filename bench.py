"""Throughput of the full sparse albedo-corrected matched-filter retrieval
(initialisation + 10 reweighting iterations) on one GB300.

Workload: a synthetic AVIRIS-NG-shaped flightline, 4000 rows x 598 detector
columns x 72 bands (2122-2488 nm) float32, 5% of pixels masked, 20 plume
blobs; lambda = 1e-3, eps = 1e-9, 10 iterations, one partition per column.
Metric: Mpixel/s = rows * cols / (seconds per retrieval), masked pixels
counted.  The headline form computes the background moments on the tensor
cores (bf16 hi + lo split, float32 accumulation); the same schedule with
float32 moments and the literal schedule of the algorithm figure (plain
FP32) are timed beside it.  Also measured: the precision form on the
20000-row, cond(C) = 1e7 workload (alpha and C errors), the batched form on
64 flightlines in one retrieval, and the differentiation form.  The FP64
oracle runs only in the CPU-baseline leg, whose outputs also give every
alpha / C error figure.  One JSON line on stdout (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import os


def cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


# the oracle's BLAS uses every host core the process may run on (set before
# numpy loads its BLAS)
for _v in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, str(cores()))

import argparse  # noqa: E402
import ctypes  # noqa: E402
import hashlib  # noqa: E402
import json  # noqa: E402
import subprocess  # noqa: E402
import sys  # noqa: E402
import tempfile  # noqa: E402
import threading  # noqa: E402
import time  # noqa: E402

import numpy as np  # noqa: E402

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOAD = "flightline-4000x598x72"
PRECISION_WORKLOAD = "precision-20000x598x72"
SMALL_WORKLOAD = "plain-512x16x72"
METRIC = "Mpixel/s full sparse-MF retrieval (10 iters) vs plain FP32 on GB300, at stated alpha error"
UNIT = "Mpixel/s"
FALLBACK_HBM_GBS = 6800.0
FALLBACK_BF16_TFLOPS = 1900.0
# the method's covariance work per pixel in the BF16-split form: three
# B x B products (H^T H, H^T L, L^T H) of 2 B^2 flop each at B = 72
METHOD_SYRK_FLOP_PER_PIXEL = 3 * 2 * 72 * 72


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def tensor_peak():
    """bf16 dense peak (TFLOP/s) for a kernel timed alone (burst figure)."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops"]), "measured (MEASURED_PEAKS.json bf16_tflops)"
    except Exception:
        return FALLBACK_BF16_TFLOPS, "fallback 1.9 PFLOP/s"


def source_hash(files):
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


# DRAM traffic of one pixel-kernel launch on this workload, from the ncu
# capture summarised in profiles/ (dram__bytes_read.sum + dram__bytes_write.sum).
# Valid only while the kernel source is unchanged (hash of the files below).
PIXEL_KERNEL_SOURCES = ["paper_2003_02978_gb300/csrc/mf_pixel.cu",
                        "paper_2003_02978_gb300/csrc/mf_pixel_body.cuh",
                        "paper_2003_02978_gb300/csrc/mf_pixel_io.cuh",
                        "paper_2003_02978_gb300/csrc/mf_tma.cuh",
                        "paper_2003_02978_gb300/csrc/mf_common.cuh"]
PIXEL_TRAFFIC_SUMMARY = os.path.join(ROOT, "profiles", "pixel_kernel_flightline-4000x598x72.md")


def pixel_traffic():
    """(bytes_per_launch, source_hash) from the committed ncu summary's
    'traffic_bytes_per_launch:' and 'source_hash:' lines, if present."""
    out = {}
    try:
        with open(PIXEL_TRAFFIC_SUMMARY) as f:
            for line in f:
                line = line.strip().strip("`").strip("- ")
                for key in ("traffic_bytes_per_launch", "source_hash"):
                    if line.startswith(key + ":"):
                        out[key] = line.split(":", 1)[1].strip()
    except OSError:
        pass
    return out


# NVML clock-event reason bits (nvml.h, nvmlClocksEventReason*)
_REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
            0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown"}


class ClockSampler:
    """SM clock and clock-event reasons sampled every ``period`` seconds
    through NVML (read-only queries; nvidia-smi if NVML cannot be loaded),
    between start() and stop()."""

    def __init__(self, device_index=0, period=0.002):
        self.dev = device_index
        self.period = period
        self.samples = []       # (sm_mhz, reasons bitmask)
        self.sm_max = None
        self._stop = threading.Event()
        self._thread = None
        self._smi = None
        self.source = None

    def _nvml_handle(self):
        nv = ctypes.CDLL("libnvidia-ml.so.1")
        if nv.nvmlInit_v2() != 0:
            raise RuntimeError("nvmlInit failed")
        h = ctypes.c_void_p()
        ok = False
        try:
            import torch
            uuid = str(torch.cuda.get_device_properties(self.dev).uuid)
            uuid = uuid if uuid.startswith("GPU-") else "GPU-" + uuid
            ok = nv.nvmlDeviceGetHandleByUUID(uuid.encode(), ctypes.byref(h)) == 0
        except Exception:
            ok = False
        if not ok and nv.nvmlDeviceGetHandleByIndex_v2(self.dev, ctypes.byref(h)) != 0:
            raise RuntimeError("no NVML handle")
        return nv, h

    def start(self):
        try:
            nv, h = self._nvml_handle()
            mx = ctypes.c_uint()
            if nv.nvmlDeviceGetMaxClockInfo(h, 1, ctypes.byref(mx)) == 0:  # NVML_CLOCK_SM
                self.sm_max = float(mx.value)
            reasons_fn = getattr(nv, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
                nv.nvmlDeviceGetCurrentClocksThrottleReasons

            def loop():
                c = ctypes.c_uint()
                r = ctypes.c_ulonglong()
                while not self._stop.is_set():
                    if nv.nvmlDeviceGetClockInfo(h, 1, ctypes.byref(c)) == 0 and \
                            reasons_fn(h, ctypes.byref(r)) == 0:
                        self.samples.append((float(c.value), int(r.value)))
                    time.sleep(self.period)
            self.source = f"NVML every {self.period * 1e3:.0f} ms"
        except Exception:
            fields = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,"
                      "clocks_event_reasons.hw_thermal_slowdown,"
                      "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
            try:
                self._smi = subprocess.Popen(
                    ["nvidia-smi", f"--id={self.dev}", f"--query-gpu={fields}",
                     "--format=csv,noheader,nounits", "-lms", "50"],
                    stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            except Exception:
                return

            def loop():
                bits = (0x8, 0x40, 0x20, 0x4)
                for ln in self._smi.stdout:
                    parts = [p.strip() for p in ln.split(",")]
                    try:
                        sm, smax = float(parts[0]), float(parts[1])
                    except (ValueError, IndexError):
                        continue
                    self.sm_max = smax
                    r = sum(b for b, v in zip(bits, parts[2:6]) if v.lower() in ("active", "1"))
                    self.samples.append((sm, r))
            self.source = "nvidia-smi every 50 ms"
        self._thread = threading.Thread(target=loop, daemon=True)
        self._thread.start()

    def stop(self):
        self._stop.set()
        if self._smi is not None:
            self._smi.terminate()
            try:
                self._smi.wait(timeout=5)
            except Exception:
                self._smi.kill()
        if self._thread is not None:
            self._thread.join(timeout=5)
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": self.sm_max, "reasons": ["no samples"],
                    "samples": 0, "source": self.source}
        sm = [s for s, _ in self.samples]
        reasons = sorted({name for _, r in self.samples for bit, name in _REASONS.items()
                          if r & bit})
        return {"sm_mhz": float(np.median(sm)), "sm_min_mhz": float(min(sm)),
                "sm_max_mhz": self.sm_max, "reasons": reasons, "samples": len(sm),
                "source": self.source, "window": "warm-up and timed steps of the headline form"}


def dist_init():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64,
                     device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------ CPU-baseline leg (oracle)
def oracle_partitions(cube, mask, k, lam, eps, n_iter):
    """The FP64 oracle on whole partitions (cube (rows, ncols, B) float32
    numpy, mask (rows, ncols)), timed: (alpha, status, seconds)."""
    import oracle
    kk = np.asarray(k, dtype=np.float32).astype(np.float64)
    t0 = time.perf_counter()
    a, st = oracle.retrieve(cube.astype(np.float64), kk, lam, eps, n_iter, mask=mask)
    return a, st, time.perf_counter() - t0


def oracle_one_thread(cube, mask, k, lam, eps, n_iter):
    """The same oracle run in a fresh interpreter whose BLAS uses one thread:
    seconds, or None if that run failed."""
    with tempfile.TemporaryDirectory() as d:
        np.save(os.path.join(d, "cube.npy"), cube)
        np.save(os.path.join(d, "mask.npy"), mask)
        np.save(os.path.join(d, "k.npy"), np.asarray(k, np.float32))
        code = ("import sys, time, numpy as np; sys.path.insert(0, %r); import oracle; "
                "d = %r; c = np.load(d + '/cube.npy').astype(np.float64); "
                "m = np.load(d + '/mask.npy'); k = np.load(d + '/k.npy').astype(np.float64); "
                "t0 = time.perf_counter(); oracle.retrieve(c, k, %r, %r, %d, mask=m); "
                "print(time.perf_counter() - t0)") % (ROOT, d, lam, eps, n_iter)
        env = dict(os.environ, OPENBLAS_NUM_THREADS="1", OMP_NUM_THREADS="1",
                   MKL_NUM_THREADS="1")
        try:
            r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True,
                               text=True, timeout=600)
            return float(r.stdout.strip().splitlines()[-1])
        except Exception:
            return None


def alpha_figures(got, ref, valid):
    """e_inf = max|got - ref| / max|ref|, e_2 = ||got - ref|| / ||ref|| over
    the valid pixels, how many differ by more than 1e-4 * max|ref|, and the
    zero-flips among those (one side exactly 0: the clamp max(0, .) of a
    near-threshold pixel went the other way, after which the reweighting's
    zero is sticky) with e_inf and e_2 over the other pixels."""
    g = np.asarray(got, np.float64)[valid]
    r = np.asarray(ref, np.float64)[valid]
    if r.size == 0:
        return {"e_inf": 0.0, "e_2": 0.0, "n_valid": 0, "n_over_1e-4": 0}
    d = np.abs(g - r)
    scale = max(np.abs(r).max(), 1e-30)
    nr = max(np.linalg.norm(r), 1e-30)
    over = d > 1e-4 * scale
    flips = over & ((g == 0) | (r == 0))
    keep = ~flips
    return {"e_inf": float(d.max() / scale), "e_2": float(np.linalg.norm(g - r) / nr),
            "n_valid": int(r.size), "n_over_1e-4": int(over.sum()),
            "n_zero_flips": int(flips.sum()),
            "e_inf_excl_flips": float(d[keep].max() / scale) if keep.any() else 0.0,
            "e_2_excl_flips": float(np.linalg.norm(d[keep]) / nr)}


def covariance_figures(cov_gpu, mu_gpu, X):
    """C^0 and mu^0 of one partition against the FP64 oracle's statistics of
    its valid pixels X: ||dC||_F / ||C||_F, the error along each eigenvector
    u of C, |u^T dC u| / lambda_u (largest, and at the smallest eigenvalue),
    cond(C) and the mean's relative error."""
    import oracle
    m = oracle.mean_vector(X)
    C = oracle.covariance_about(X - m)
    ev, V = np.linalg.eigh(C)
    dC = cov_gpu - C
    eig = np.abs(np.einsum("bi,bc,ci->i", V, dC, V)) / ev
    return {"c_fro": float(np.linalg.norm(dC) / np.linalg.norm(C)),
            "c_eig_max": float(eig.max()), "c_eig_at_min": float(eig[0]),
            "cond": float(ev[-1] / ev[0]),
            "mu_rel": float(np.abs(mu_gpu - m).max() / np.abs(m).max())}


def run_reference(args, world, rank):
    """The FP64 CPU oracle timed as the reference arm (host cores)."""
    if rank != 0:
        return
    from synth import workload_scene
    sc, prm = workload_scene(WORKLOAD, seed=0, device="cpu")
    rows = sc.cube.shape[0]
    rng = np.random.default_rng(123)
    # whole partitions per step: 6 (about half a second of oracle work on
    # 8-16 cores), fewer for long runs so that warm-up + K steps stay within
    # a couple of minutes
    ncol = max(1, min(6, 1200 // max(1, args.steps + args.warmup)))
    cube = sc.cube.numpy()
    mask = sc.mask.numpy()
    times = []
    for step in range(args.warmup + args.steps):
        cols = np.sort(rng.choice(cube.shape[1], size=ncol, replace=False))
        _, _, dt = oracle_partitions(cube[:, cols], mask[:, cols], sc.k, prm["lam"], prm["eps"],
                                     prm["n_iter"])
        if step >= args.warmup:
            times.append(dt)
    value = rows * ncol / float(np.mean(times)) / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": float(np.mean(times)) * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "rows": rows, "cols": 598, "bands": 72,
                       "n_iter": prm["n_iter"], "lambda": prm["lam"], "eps": prm["eps"],
                       "sample": f"{ncol} random whole partitions ({ncol} x {rows} pixels) per step"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores(), "kind": "oracle",
                             "blas_threads": int(os.environ.get("OPENBLAS_NUM_THREADS", "0")),
                             "sample": f"{ncol} whole partitions of {rows} rows per step"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------- GPU measurements
def time_retrievals(plan, args_fn, steps, warmup, dev, world=1, stream=None):
    """ms per retrieval over `steps` calls after `warmup` calls, CUDA events on
    the launching stream, barrier + synchronize on both sides."""
    import torch
    for _ in range(warmup):
        args_fn(plan)
    torch.cuda.synchronize(dev)
    barrier(world)
    torch.cuda.synchronize(dev)
    s = stream if stream is not None else torch.cuda.current_stream(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(s)
    for _ in range(steps):
        args_fn(plan)
    e1.record(s)
    torch.cuda.synchronize(dev)
    barrier(world)
    return e0.elapsed_time(e1) / steps


def precision_form(dev, n_cols=8):
    """The precision workload (20000 x 598 x 72, cond(C_bg) = 1e7, SNR
    100-500, 10 iterations) in the BF16-split and float32 forms: Mpixel/s and,
    for sampled whole partitions, alpha and the initial statistics (for the
    oracle comparison of the CPU-baseline leg)."""
    import torch
    import paper_2003_02978_gb300 as mfg
    from synth import workload_scene
    sc, prm = workload_scene(PRECISION_WORKLOAD, seed=0, device=dev)
    rows, cols, bands = sc.cube.shape
    k = torch.as_tensor(np.asarray(sc.k, np.float32), device=dev)
    out = torch.empty((rows, cols), dtype=torch.float32, device=dev)
    cols_s = np.unique(np.concatenate([np.random.default_rng(5).choice(cols, n_cols - 2,
                                                                     replace=False),
                                       [0, cols - 1]]))
    res = {"workload": f"{PRECISION_WORKLOAD}: cond(C_bg) 1e7, SNR 100-500, "
                       f"n_iter {prm['n_iter']}, lambda {prm['lam']}, 5% masked",
           "pixels": rows * cols, "forms": {}}
    keep = {"cols": cols_s, "cube": sc.cube[:, cols_s].cpu().numpy(),
            "mask": sc.mask[:, cols_s].cpu().numpy(), "k": sc.k, "prm": prm, "forms": {}}

    def run(plan):
        plan.retrieve(sc.cube, k, prm["lam"], prm["eps"], prm["n_iter"], mask=sc.mask, out=out)

    for name, prec, flags in (("bf16split_fused", mfg.BF16SPLIT, mfg.ALBEDO | mfg.SPARSE),
                              ("fp32_fused", mfg.FP32, mfg.ALBEDO | mfg.SPARSE),
                              ("plain_fp32_literal", mfg.FP32,
                               mfg.ALBEDO | mfg.SPARSE | mfg.LITERAL)):
        plan = mfg.Plan(rows, cols, bands, flags=flags, precision=prec)
        ms = time_retrievals(plan, run, 10, 3, dev)
        status_ok = bool(np.all(plan.status() == 0))
        mu, cov = plan.background()
        keep["forms"][name] = {"alpha": out[:, cols_s].cpu().numpy(),
                               "mu": mu[cols_s].cpu().numpy(), "cov": cov[cols_s].cpu().numpy()}
        res["forms"][name] = {"value": rows * cols / (ms * 1e-3) / 1e6, "ms_per_retrieval": ms,
                              "status_ok": status_ok}
        plan.close()
        del mu, cov
    del sc, out
    torch.cuda.empty_cache()
    return res, keep


BATCH_LINES = 64


def persistent_only(args, mfg, run, shape, dev, world, stream):
    """The headline workload (BF16-split statistics, fused iterations) in the
    persistent work-queue schedule: pilot, statistics, then one queue_kernel
    launch per retrieval, replayed as a CUDA graph.  Prints one JSON line of
    its own (not the bench contract's line)."""
    rows, cols, bands = shape
    plan = mfg.Plan(rows, cols, bands, flags=mfg.ALBEDO | mfg.SPARSE | mfg.PERSISTENT,
                    precision=mfg.BF16SPLIT)
    run(plan)
    ms = time_retrievals(plan, run, args.steps, args.warmup, dev, world, stream)
    plan.timeline(True)
    run(plan)
    plan.timeline_read()
    run(plan)
    spans = plan.timeline_read()
    plan.timeline(False)
    ok = bool(np.all(plan.status() == 0))
    plan.close()
    print(json.dumps({"workload": WORKLOAD, "schedule": "persistent work queue (MF_PERSISTENT)",
                      "value": rows * cols / (ms * 1e-3) / 1e6, "unit": "Mpixel/s",
                      "ms_per_step": ms, "steps": args.steps, "status_ok": ok,
                      "launches_per_retrieval": [[kd, round(t1 - t0, 1)] for kd, t0, t1 in spans]}),
          flush=True)


def batched_form(dev, precision, n_lines=BATCH_LINES):
    """The batched workload: `n_lines` flightlines (rows uniform in
    2000-30000, 598 x 72, per-column masked fraction U(0, 0.3), per-line
    n_iter in 5..20 and lambda log-uniform in [1e-4, 1e-2]; one shared target
    spectrum), drawn straight into one preallocated stacked cube, retrieved in
    one batched call (CUDA-graph replay, launch shapes from the autotuner),
    against the plain FP32 form (literal schedule, one single-line plan per
    line, timed line by line).  Returns the figures and sampled partitions of
    three lines with both sides' alpha, for the oracle comparison."""
    import torch
    import paper_2003_02978_gb300 as mfg
    from paper_2003_02978_gb300 import tune
    from synth import batched_lines, make_scene
    lines = batched_lines(n_lines, seed=11)
    rows = [ln["rows"] for ln in lines]
    lams = [ln["lam"] for ln in lines]
    nits = [ln["n_iter"] for ln in lines]
    R, cols, bands = sum(rows), 598, 72
    cube = torch.empty((R, cols, bands), dtype=torch.float32, device=dev)
    mask = torch.empty((R, cols), dtype=torch.uint8, device=dev)
    r0 = 0
    k_np = None
    for ln in lines:
        r1 = r0 + ln["rows"]
        sc = make_scene(ln["rows"], cols, bands, n_plumes=20, plume_sigma=(3.0, 15.0),
                        plume_peak=(500.0, 5000.0), mask_col_frac=ln["mask_col_frac"],
                        seed=ln["seed"], device=dev, keep_truth=False, out=cube[r0:r1],
                        mask_out=mask[r0:r1])
        if k_np is None:
            k_np = np.asarray(sc.k, np.float32)
        del sc
        r0 = r1
    k = torch.as_tensor(k_np, device=dev)
    npix = R * cols
    t0 = time.perf_counter()
    # shapes for both schedules: the persistent one gains from longer pixel
    # items (fewer items to take and wait for)
    tuned = []
    tuning = tune.autotune(cube, k, lams, 1e-9, nits, mask=mask, line_rows=rows,
                           precision=precision, reps=1, use_cache=False,
                           candidates=[(0, 0, 0), (256, 0, 0), (1024, 0, 0), (0, 512, 0),
                                       (256, 512, 0), (1024, 512, 0), (0, 0, 1), (1024, 0, 1),
                                       (2048, 0, 1), (4096, 0, 1)], results_out=tuned)
    tune_s = time.perf_counter() - t0
    plan = mfg.BatchPlan(rows, cols, bands, precision=precision, tuning=tuning)
    out = torch.empty((R, cols), dtype=torch.float32, device=dev)

    def run(pl):
        pl.retrieve(cube, k, lams, 1e-9, nits, mask=mask, out=out)

    ms_b = time_retrievals(plan, run, 3, 2, dev)
    status_ok = bool(np.all(plan.status() == 0))
    slices = plan.line_slices()
    plan.close()
    # the other schedule, one launch per pass (a CUDA graph of ~2 n_iter
    # launches) or the persistent work queue (one launch after the
    # statistics): timed at its own best shapes, and run once at the chosen
    # shapes, where the arithmetic is the same, to check bit-identical alpha
    other_p = 0 if tuning.get("persistent") else 1
    other = min((r for r in tuned if r[1]["persistent"] == other_p), key=lambda r: r[0])[1]
    out_o = torch.empty_like(out)

    def run_o(pl):
        pl.retrieve(cube, k, lams, 1e-9, nits, mask=mask, out=out_o)

    plan_o = mfg.BatchPlan(rows, cols, bands, precision=precision, tuning=other)
    ms_o = time_retrievals(plan_o, run_o, 3, 2, dev)
    plan_o.close()
    plan_s = mfg.BatchPlan(rows, cols, bands, precision=precision,
                           tuning=dict(tuning, persistent=other_p))
    run_o(plan_s)
    torch.cuda.synchronize(dev)
    same_bits = bool(torch.equal(out.view(torch.int32), out_o.view(torch.int32)))
    plan_s.close()
    del out_o
    ms_seq, ms_queue = (ms_o, ms_b) if tuning.get("persistent") else (ms_b, ms_o)
    tuning_seq, tuning_queue = (other, tuning) if tuning.get("persistent") else (tuning, other)
    # plain FP32 form: literal schedule, one plan per line
    outp = torch.empty_like(out)
    ms_p = 0.0
    for sl, lam, n in zip(slices, lams, nits):
        pl_ = mfg.Plan(sl.stop - sl.start, cols, bands, flags=mfg.ALBEDO | mfg.SPARSE | mfg.LITERAL)
        cv, mv, ov = cube[sl], mask[sl], outp[sl]

        def run_p(p_, cv=cv, mv=mv, ov=ov, lam=lam, n=n):
            p_.retrieve(cv, k, lam, 1e-9, n, mask=mv, out=ov)
        ms_p += time_retrievals(pl_, run_p, 1, 1, dev)
        pl_.close()
    # sampled partitions of the first, a middle and the last line
    rng = np.random.default_rng(3)
    samples = []
    for li in (0, n_lines // 2, n_lines - 1):
        sl = slices[li]
        c = np.sort(rng.choice(cols, 2, replace=False))
        samples.append({"line": li, "rows": sl.stop - sl.start, "cols": c,
                        "lam": lams[li], "n_iter": nits[li],
                        "cube": cube[sl][:, c].cpu().numpy(), "mask": mask[sl][:, c].cpu().numpy(),
                        "batched": out[sl][:, c].cpu().numpy(),
                        "plain": outp[sl][:, c].cpu().numpy()})
    del cube, mask, out, outp
    torch.cuda.empty_cache()
    res = {"workload": f"{n_lines} flightlines ({npix / 1e6:.1f} Mpixel, {R} rows in all), "
                       "rows U(2000, 30000), 598 x 72, per-column masked fraction U(0, 0.3), "
                       "n_iter U{5..20}, lambda log-U(1e-4, 1e-2)",
           "lines": n_lines, "pixels": npix, "cube_gb": R * cols * bands * 4 / 1e9,
           "precision": "bf16split" if precision else "fp32",
           "tuning": tuning, "autotune_s": tune_s,
           "value": npix / (ms_b * 1e-3) / 1e6, "ms_per_batch": ms_b,
           "schedule": "persistent work queue" if tuning.get("persistent") else "launch per pass",
           "launch_per_pass_value": npix / (ms_seq * 1e-3) / 1e6,
           "launch_per_pass_tuning": tuning_seq,
           "persistent_value": npix / (ms_queue * 1e-3) / 1e6,
           "persistent_tuning": tuning_queue,
           "schedules_bit_identical_at_equal_shapes": same_bits,
           "plain_fp32_value": npix / (ms_p * 1e-3) / 1e6, "plain_fp32_ms": ms_p,
           "status_ok": status_ok}
    return res, {"k": k_np, "samples": samples}


def differentiation_form(dev):
    """Forward with checkpoints and the backward pass (gradients for s, lambda
    and the cube) on the differentiation workload (8000 x 598 x 72, 10
    iterations, loss = MSE of alpha against the injected plume map), timed
    with CUDA events; the target is backward <= 3 x forward."""
    import torch
    import paper_2003_02978_gb300 as mfg
    from synth import workload_scene
    sc, prm = workload_scene("diff-8000x598x72", seed=3, device=dev)
    rows, cols, bands = sc.cube.shape
    k = torch.as_tensor(np.asarray(sc.k, np.float32), device=dev)
    plan = mfg.Plan(rows, cols, bands)
    ck = torch.empty(plan.ckpt_bytes(prm["n_iter"], True) + 256, dtype=torch.uint8, device=dev)
    truth = torch.as_tensor(sc.alpha_true, dtype=torch.float32, device=dev)
    e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    fw, bw_ = [], []
    for it in range(4):
        e[0].record()
        alpha, _ = plan.retrieve_train(sc.cube, k, prm["lam"], prm["eps"], prm["n_iter"],
                                       mask=sc.mask, cube_grad=True, ckpt=ck)
        e[1].record()
        g = 2.0 * (alpha - truth) / alpha.numel()
        e[2].record()
        plan.backward(ck, g, cube_grad=True)
        e[3].record()
        torch.cuda.synchronize()
        if it >= 1:
            fw.append(e[0].elapsed_time(e[1]))
            bw_.append(e[2].elapsed_time(e[3]))
    out = torch.empty((rows, cols), dtype=torch.float32, device=dev)

    def run(pl):
        pl.retrieve(sc.cube, k, prm["lam"], prm["eps"], prm["n_iter"], mask=sc.mask, out=out)
    f_plain = time_retrievals(plan, run, 5, 3, dev)
    st_ok = bool(np.all(plan.status() == 0))
    plan.close()
    del ck, sc
    torch.cuda.empty_cache()
    f_ms, b_ms = float(np.median(fw)), float(np.median(bw_))
    return {"workload": f"diff-{rows}x{cols}x{bands}, n_iter {prm['n_iter']}, MSE loss, "
                        "gradients for s, lambda and the cube",
            "forward_ckpt_ms": f_ms, "forward_ms": f_plain, "backward_ms": b_ms,
            "backward_over_forward": b_ms / f_plain, "status_ok": st_ok}


def cpu_leg(sc, prm, alphas, precision_keep, batched_keep):
    """The oracle's part of the bench (rank 0, N = 1 only): its throughput on
    a bounded sample of the benchmark workload with every host core and with
    one BLAS thread, on the small workload in full, and its outputs, which
    give the alpha and C errors of every GPU form measured."""
    import oracle
    from synth import workload_scene
    rows, cols, _ = sc.cube.shape
    cols_s = np.sort(np.random.default_rng(7).choice(cols, size=8, replace=False))
    cube_s = sc.cube[:, cols_s, :].cpu().numpy()
    mask_s = sc.mask[:, cols_s].cpu().numpy()
    ref, _, dt = oracle_partitions(cube_s, mask_s, sc.k, prm["lam"], prm["eps"], prm["n_iter"])
    valid = oracle.valid_pixels(cube_s, mask_s)
    amp = oracle.retrieve_amplification(cube_s.astype(np.float64),
                                        np.asarray(sc.k, np.float32).astype(np.float64),
                                        prm["lam"], prm["eps"], prm["n_iter"], mask=mask_s)
    err = {}
    for name, a in alphas.items():
        f = alpha_figures(a[:, cols_s], ref, valid)
        f["n_amp_over_10"] = int((amp[valid] > 10).sum())
        f["max_amp"] = float(amp[valid].max())
        err[name] = f
    dt1 = oracle_one_thread(cube_s, mask_s, sc.k, prm["lam"], prm["eps"], prm["n_iter"])
    sm, sprm = workload_scene(SMALL_WORKLOAD, seed=0)
    _, _, dts = oracle_partitions(sm.cube.numpy(), None, sm.k, sprm["lam"], sprm["eps"],
                                  sprm["n_iter"])
    npx = rows * len(cols_s)
    cpu = {"value": npx / dt / 1e6, "unit": UNIT, "cores": cores(), "kind": "oracle",
           "blas_threads": int(os.environ.get("OPENBLAS_NUM_THREADS", "0")),
           "sample": f"{len(cols_s)} whole partitions x {rows} rows of {WORKLOAD}",
           "one_thread": None if dt1 is None else {"value": npx / dt1 / 1e6, "blas_threads": 1,
                                                   "sample": "the same"},
           "small_workload_full": {"workload": SMALL_WORKLOAD,
                                   "value": 512 * 16 / dts / 1e6, "seconds": dts}}
    prec = None
    if precision_keep is not None:
        kp = precision_keep
        p = kp["prm"]
        ref3, st3, _ = oracle_partitions(kp["cube"], kp["mask"], kp["k"], p["lam"], p["eps"],
                                         p["n_iter"])
        v3 = oracle.valid_pixels(kp["cube"], kp["mask"])
        prec = {}
        for name, f in kp["forms"].items():
            cf = [covariance_figures(f["cov"][j], f["mu"][j],
                                     kp["cube"][v3[:, j], j].astype(np.float64))
                  for j in range(len(kp["cols"]))]
            prec[name] = {"alpha": alpha_figures(f["alpha"], ref3, v3),
                          "c_fro": max(c["c_fro"] for c in cf),
                          "c_eig_max": max(c["c_eig_max"] for c in cf),
                          "c_eig_at_min": max(c["c_eig_at_min"] for c in cf),
                          "mu_rel": max(c["mu_rel"] for c in cf),
                          "cond_c0": [min(c["cond"] for c in cf), max(c["cond"] for c in cf)]}
        prec["sample"] = f"{len(kp['cols'])} whole partitions x {kp['cube'].shape[0]} rows"
    bat = None
    if batched_keep is not None:
        bat = {"lines": []}
        for s in batched_keep["samples"]:
            r, _, _ = oracle_partitions(s["cube"], s["mask"], batched_keep["k"], s["lam"], 1e-9,
                                        s["n_iter"])
            v = oracle.valid_pixels(s["cube"], s["mask"])
            bat["lines"].append({"line": s["line"], "rows": s["rows"], "n_iter": s["n_iter"],
                                 "lambda": s["lam"],
                                 "batched": alpha_figures(s["batched"], r, v),
                                 "plain_fp32": alpha_figures(s["plain"], r, v)})
        bat["sample"] = "2 whole partitions of the first, a middle and the last line"
    return cpu, err, prec, bat


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--no-oracle", action="store_true", help="skip the CPU-baseline leg")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched form")
    ap.add_argument("--no-diff", action="store_true", help="skip the differentiation form")
    ap.add_argument("--no-precision", action="store_true", help="skip the precision form")
    ap.add_argument("--batch-lines", type=int, default=BATCH_LINES)
    ap.add_argument("--persistent-only", action="store_true",
                    help="time only the headline workload in the persistent work-queue schedule "
                         "(MF_PERSISTENT) and print its own line (for profiling that kernel)")
    args = ap.parse_args()
    world, rank, local = dist_init()
    if args.impl == "reference":
        run_reference(args, world, rank)
        return
    assert args.warmup >= 3, "at least 3 warm-up steps"

    import torch
    import paper_2003_02978_gb300 as mfg
    from paper_2003_02978_gb300 import build as _build
    from synth import workload_scene

    _build.build()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    sc, prm = workload_scene(WORKLOAD, seed=rank, device=dev)
    rows, cols, bands = sc.cube.shape
    npix = rows * cols
    n_iter = prm["n_iter"]
    k = torch.as_tensor(np.asarray(sc.k, np.float32), device=dev)
    out = torch.empty((rows, cols), dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def run(plan):
        plan.retrieve(sc.cube, k, prm["lam"], prm["eps"], n_iter, mask=sc.mask, out=out)

    if args.persistent_only:
        persistent_only(args, mfg, run, sc.cube.shape, dev, world, stream)
        return

    # --- headline form: fused schedule, moments on the tensor cores (bf16
    # hi + lo split, float32 accumulation), float32 pixel path, double-float
    # solves; one CUDA-graph launch per retrieval; clocks sampled over the
    # warm-up and timed steps
    plan = mfg.Plan(rows, cols, bands, flags=mfg.ALBEDO | mfg.SPARSE, precision=mfg.BF16SPLIT)
    run(plan)  # first call: graph capture
    torch.cuda.synchronize(dev)
    clk = ClockSampler(local)
    clk.start()
    ms = time_retrievals(plan, run, args.steps, args.warmup, dev, world, stream)
    clocks = clk.stop()
    ms_max = max_over_ranks(ms, world)
    value = world * npix / (ms_max * 1e-3) / 1e6
    alphas = {"bf16split_fused": out.cpu().numpy()}

    # --- the same fused schedule with float32 (SIMT) moments
    plan_f32 = mfg.Plan(rows, cols, bands, flags=mfg.ALBEDO | mfg.SPARSE)
    f32_steps = max(2, args.steps // 4)
    ms_f32 = time_retrievals(plan_f32, run, f32_steps, args.warmup, dev, world, stream)
    alphas["fp32_fused"] = out.cpu().numpy()

    # --- plain FP32 form (literal schedule of the algorithm figure)
    plan_lit = mfg.Plan(rows, cols, bands, flags=mfg.ALBEDO | mfg.SPARSE | mfg.LITERAL)
    lit_steps = max(2, args.steps // 8)
    ms_lit = time_retrievals(plan_lit, run, lit_steps, args.warmup, dev, world, stream)
    alphas["plain_fp32_literal"] = out.cpu().numpy()

    # --- per-kernel device time: direct launches (no graph) with CUDA events
    # around every kernel on the launching stream
    prof_steps = max(20, args.steps // 4)

    def profiled(pl, steps):
        for _ in range(2):
            run(pl)
        torch.cuda.synchronize(dev)
        pl.profile(True)
        pl.profile_read()
        for _ in range(steps):
            run(pl)
        prof = pl.profile_read()
        pl.profile(False)
        return prof

    prof = profiled(plan, prof_steps)

    # --- the same split inside the timed configuration (one CUDA graph per
    # retrieval): the library's device timeline, each launch from its first
    # CTA's start to its last CTA's end on the GPU's global timer
    def timeline(pl, steps):
        pl.timeline(True)
        run(pl)  # re-captures the graph with the probes
        pl.timeline_read()
        runs = []
        for _ in range(steps):
            run(pl)
            runs.append(pl.timeline_read())
        pl.timeline(False)
        run(pl)  # and back to the probe-free graph
        torch.cuda.synchronize(dev)
        return runs

    tl_runs = timeline(plan, prof_steps)
    tl_sum = {"stats": 0.0, "pixel": 0.0, "solve": 0.0}
    tl_n = {"stats": 0, "pixel": 0, "solve": 0}
    tl_span = 0.0
    for spans in tl_runs:
        for kind, t0, t1 in spans:
            if t0 is not None:
                tl_sum[kind] += t1 - t0
                tl_n[kind] += 1
        tl_span += max(t1 for _, _, t1 in spans if t1 is not None)
    nrun = len(tl_runs)
    in_graph = {kk: tl_sum[kk] / nrun for kk in tl_sum}
    in_graph["span"] = tl_span / nrun
    in_graph["gaps"] = in_graph["span"] - (in_graph["stats"] + in_graph["pixel"] +
                                           in_graph["solve"])
    in_graph["launches_per_retrieval"] = {kk: tl_n[kk] / nrun for kk in tl_n}
    in_graph["retrievals"] = nrun
    in_graph["timing"] = ("device timeline of graph replays of the headline plan: per launch "
                          "the first CTA's start to the last CTA's end (GPU global timer), "
                          "summed per kernel kind; us per retrieval")
    px_tl_s = tl_sum["pixel"] / tl_n["pixel"] * 1e-6
    f32_prof_steps = max(2, f32_steps // 2)
    prof_f32 = profiled(plan_f32, f32_prof_steps)
    px_ms, px_n = prof["pixel"]
    st_ms, st_n = prof["stats"]
    sv_ms, sv_n = prof["solve"]
    # our kernels per retrieval (the statistics mark also covers the pilot
    # kernel of the tensor-core form) x the timed retrievals
    per_step = (px_n + 2 * st_n + sv_n) / prof_steps
    launches = int(round(per_step * args.steps))
    nmask = 1 if sc.mask is not None else 0
    per_launch = [npix * (4 * bands + 4 + nmask)] + [npix * (4 * bands + 8 + nmask)] * n_iter
    alg_bytes = float(np.mean(per_launch))
    px_avg_s = px_ms / px_n * 1e-3
    hbm, peak_kind = peaks()
    achieved = alg_bytes / px_avg_s / 1e9
    cur_hash = source_hash(PIXEL_KERNEL_SOURCES)
    tr = pixel_traffic()
    traffic = float(tr["traffic_bytes_per_launch"]) if tr.get("source_hash") == cur_hash and \
        "traffic_bytes_per_launch" in tr else None

    # tensor-core statistics kernel: the method's work (three B x B products
    # per pixel) against the bf16 peak; the executed MMA work (two
    # tcgen05.mma per 16 pixels, M 128 x N 2 NP and M 128 x N NP, K 16, NP
    # the padded augmented width) stated beside it
    tc_peak, tc_src = tensor_peak()
    st_s = st_ms / st_n * 1e-3
    np_w = ((bands + 3 + 3) // 4 * 4 + 15) // 16 * 16
    method_tflops = 3 * 2 * bands * bands * npix / st_s / 1e12
    mma_tflops = 2.0 * 128 * (3 * np_w) * npix / st_s / 1e12
    st_gbs = npix * (4 * bands + 1) / st_s / 1e9
    syrk = {"kernel": "stats_tc_kernel (with its pilot kernel)", "launches": int(st_n),
            "avg_launch_us": st_s * 1e6,
            "method_flop_per_pixel": 3 * 2 * bands * bands,
            "tensor_tflops": method_tflops, "tensor_peak_tflops": tc_peak,
            "tensor_frac": method_tflops / tc_peak, "tensor_peak_source": tc_src,
            "executed_mma_flop_per_pixel": 2 * 128 * 3 * np_w,
            "executed_mma_tflops": mma_tflops, "executed_mma_frac": mma_tflops / tc_peak,
            "hbm_gbs": st_gbs, "hbm_frac": st_gbs / hbm,
            "in_graph_us": in_graph["stats"],
            "in_graph_hbm_frac": npix * (4 * bands + 1) / (in_graph["stats"] * 1e-6) / 1e9 / hbm}

    # --- end to end through the host-buffer entry point (pinned memory)
    cube_h = sc.cube.cpu().pin_memory()
    mask_h = sc.mask.cpu().pin_memory()
    k_h = np.asarray(sc.k, np.float32)
    alpha_h = torch.empty((rows, cols), dtype=torch.float32).pin_memory()
    for _ in range(2):
        plan.retrieve_host(cube_h, k_h, prm["lam"], prm["eps"], n_iter, mask=mask_h, out=alpha_h)
    e2e_steps = max(3, args.steps // 4)
    barrier(world)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        plan.retrieve_host(cube_h, k_h, prm["lam"], prm["eps"], n_iter, mask=mask_h, out=alpha_h)
    e2e_sync_s = max_over_ranks((time.perf_counter() - t0) / e2e_steps, world)
    # the same steps as a stream of cubes through mf_retrieve_host_async:
    # two staging slots, step n + 1's copy in overlapping step n's retrieval;
    # every step still copies its cube in and its alpha out, and the timed
    # region ends with the last step's alpha on the host
    outs = [torch.empty((rows, cols), dtype=torch.float32).pin_memory() for _ in range(2)]
    for i in range(2):
        plan.retrieve_host_async(cube_h, k_h, prm["lam"], prm["eps"], n_iter, mask=mask_h,
                                 out=outs[i], stream=stream)
    torch.cuda.synchronize(dev)
    barrier(world)
    t0 = time.perf_counter()
    for i in range(e2e_steps):
        plan.retrieve_host_async(cube_h, k_h, prm["lam"], prm["eps"], n_iter, mask=mask_h,
                                 out=outs[i & 1], stream=stream)
    stream.synchronize()
    e2e_s = max_over_ranks((time.perf_counter() - t0) / e2e_steps, world)
    async_matches = bool(torch.equal(outs[(e2e_steps - 1) & 1], alpha_h))
    h2d = cube_h.numel() * 4 + mask_h.numel() + k_h.size * 4
    d2h = alpha_h.numel() * 4
    plan.close()
    plan_f32.close()
    plan_lit.close()
    del cube_h, mask_h, alpha_h, outs

    precision = precision_keep = None
    batched = batched_keep = None
    differentiation = None
    if rank == 0:
        if not args.no_precision:
            precision, precision_keep = precision_form(dev)
        if not args.no_diff:
            differentiation = differentiation_form(dev)
        if not args.no_batched:
            batched, batched_keep = batched_form(dev, mfg.BF16SPLIT, args.batch_lines)

    if rank == 0:
        cpu = err = None
        if not args.no_oracle and world == 1:
            cpu, err, perr, berr = cpu_leg(sc, prm, alphas, precision_keep, batched_keep)
            if precision is not None and perr is not None:
                for name, f in perr.items():
                    if name in precision["forms"]:
                        precision["forms"][name]["errors"] = f
                precision["error_sample"] = perr.get("sample")
            if batched is not None and berr is not None:
                batched["alpha_error"] = berr
        err = err or {}
        kernels_f32 = {kk: v[0] / f32_prof_steps for kk, v in prof_f32.items()}
        result = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 (moments: bf16 hi+lo products, f32 accumulation)",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "rows": rows, "cols": cols, "bands": bands,
                       "n_iter": n_iter, "lambda": prm["lam"], "eps": prm["eps"],
                       "mask_frac": 0.05, "partitions": cols,
                       "form": "fused schedule; moments on tcgen05 tensor cores from bf16 "
                               "hi+lo split with f32 accumulation; float32 pixel path; "
                               "double-float Cholesky and solves",
                       "l2": "inputs larger than L2 (689 MB cube per step)",
                       "parallelism": f"replicas x{world}"},
            "roofline": {"kernel": "pixel_kernel", "bound": "hbm", "achieved": achieved,
                         "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                         "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)"
                         if peak_kind == "measured" else "fallback 6.8 TB/s",
                         "traffic": traffic,
                         "alg_bytes_per_launch": alg_bytes,
                         "avg_launch_us": px_avg_s * 1e6, "launches": int(px_n),
                         "timing": "CUDA events around each launch, direct launches",
                         "in_graph": {"avg_launch_us": px_tl_s * 1e6,
                                      "achieved": alg_bytes / px_tl_s / 1e9,
                                      "frac": alg_bytes / px_tl_s / 1e9 / hbm,
                                      "launches": tl_n["pixel"],
                                      "timing": "device timeline of the graph replays"}},
            "kernels_ms_per_step": {"stats": st_ms / prof_steps, "pixel": px_ms / prof_steps,
                                    "solve": sv_ms / prof_steps,
                                    "timing": "direct launches with CUDA events around every "
                                              "kernel (the headline replays a CUDA graph)"},
            "kernels_us_in_graph": in_graph,
            "gpu_launches": launches,
            "syrk": syrk,
            "forms": {"bf16split_fused": {"value": value, "ms_per_step": ms_max,
                                          "alpha_error": err.get("bf16split_fused")},
                      "fp32_fused": {"value": world * npix / (ms_f32 * 1e-3) / 1e6,
                                     "ms_per_step": ms_f32,
                                     "kernels_ms_per_step_direct": kernels_f32,
                                     "alpha_error": err.get("fp32_fused")},
                      "plain_fp32_literal": {"value": world * npix / (ms_lit * 1e-3) / 1e6,
                                             "ms_per_step": ms_lit,
                                             "alpha_error": err.get("plain_fp32_literal")}},
            "alpha_error": err.get("bf16split_fused"),
            "e2e": {"value": world * npix / e2e_s / 1e6, "unit": UNIT,
                    "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                    "api": "mf_retrieve_host_async (pinned host buffers, two device staging "
                           "slots: step n + 1's copy in overlaps step n's retrieval; host clock "
                           "from the first call to the last alpha on the host)",
                    "alpha_matches_sync": async_matches,
                    "sync": {"value": world * npix / e2e_sync_s / 1e6,
                             "api": "mf_retrieve_host (copy in, retrieve, copy out, "
                                    "synchronise, per step)"}},
            "cpu_baseline": cpu,
            "precision": precision,
            "batched": batched,
            "differentiation": differentiation,
            "clocks": clocks,
        }
        print(json.dumps(result), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
