"""Autotuner of the launch shapes of a plan (rows per pixel-kernel CTA, rows
per statistics work item) and of its schedule (a launch per pass, or the
persistent work queue of MF_PERSISTENT), with a JSON cache.

For a shape (columns, bands, line lengths, precision, flags) it times a few
candidate shapes on the caller's own cube with CUDA events (one warm-up and
``reps`` timed retrievals each, every candidate a fresh plan) and keeps the
fastest; results are cached per GPU model in a JSON file (``MF_TUNE_CACHE``,
default ``~/.cache/paper_2003_02978_gb300/tune.json``).  Every candidate runs
the same kernels and arithmetic: only the grid decomposition differs.
"""
from __future__ import annotations

import json
import os
from pathlib import Path

import torch

from . import BatchPlan, Plan

PIXEL_ROWS = (0, 128, 256, 384, 768)
STAT_ROWS = (0, 512, 2048)


def cache_path() -> Path:
    p = os.environ.get("MF_TUNE_CACHE")
    return Path(p) if p else Path.home() / ".cache" / "paper_2003_02978_gb300" / "tune.json"


def _key(line_rows, cols, bands_total, band_lo, band_hi, col_group, flags, precision):
    gpu = torch.cuda.get_device_name() if torch.cuda.is_available() else "none"
    rows = sorted(int(r) for r in line_rows)
    # lines bucketed by count and total rows (within 2x), so that similar
    # batches share an entry
    total = sum(rows)
    bucket = 1 << max(0, total.bit_length() - 1)
    return (f"{gpu}|cols={cols}|bands={bands_total}[{band_lo}:{band_hi}]|g={col_group}"
            f"|flags={flags}|prec={precision}|lines={len(rows)}|rows~{bucket}")


def load_cache() -> dict:
    try:
        return json.loads(cache_path().read_text())
    except (OSError, ValueError):
        return {}


def save_cache(c: dict) -> None:
    p = cache_path()
    p.parent.mkdir(parents=True, exist_ok=True)
    tmp = p.with_suffix(".tmp")
    tmp.write_text(json.dumps(c, indent=1, sort_keys=True))
    tmp.replace(p)


def _time(plan, cube, k, lam, eps, n_iter, mask, reps):
    out = torch.empty((cube.shape[0], cube.shape[1]), dtype=torch.float32, device=cube.device)
    plan.retrieve(cube, k, lam, eps, n_iter, mask=mask, out=out)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        plan.retrieve(cube, k, lam, eps, n_iter, mask=mask, out=out)
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def autotune(cube, k, lam, eps, n_iter, mask=None, line_rows=None, band_lo=0, band_hi=None,
             col_group=1, flags=3, precision=0, reps=3, use_cache=True, verbose=False,
             candidates=None, results_out=None):
    """Best {pixel_rows, stat_rows, persistent} for this cube's shape (a dict
    for the ``tuning`` argument of Plan / BatchPlan), timing candidates on the
    cube.  ``candidates``: optional (pixel_rows, stat_rows[, persistent])
    tuples to try instead of the full grid PIXEL_ROWS x STAT_ROWS (launch per
    pass) plus the default shapes in the persistent schedule.  ``results_out``:
    a list that receives every timed candidate as (ms, tuning)."""
    rows, cols, bt = cube.shape
    band_hi = bt if band_hi is None else band_hi
    line_rows = [rows] if line_rows is None else list(line_rows)
    key = _key(line_rows, cols, bt, band_lo, band_hi, col_group, flags, precision)
    cache = load_cache() if use_cache else {}
    if key in cache:
        return dict(cache[key]["tuning"])
    if candidates is None:
        candidates = [(pr, sr, 0) for pr in PIXEL_ROWS for sr in STAT_ROWS] + [(0, 0, 1)]
    candidates = [tuple(c) + (0,) * (3 - len(c)) for c in candidates]
    # the BF16-split bound is stated up to 1024 rows per statistics item; the
    # persistent schedule runs the fused iterations only
    candidates = [(pr, sr, pq) for pr, sr, pq in candidates
                  if not (precision == 1 and sr > 1024) and not (pq and flags & 4)]
    results = []
    for pr, sr, pq in candidates:
        t = {"pixel_rows": pr, "stat_rows": sr, "persistent": pq}
        if len(line_rows) == 1:
            plan = Plan(rows, cols, bt, band_lo, band_hi, col_group, flags, precision,
                        tuning=t)
        else:
            plan = BatchPlan(line_rows, cols, bt, band_lo, band_hi, col_group, flags,
                             precision, tuning=t)
        ms = _time(plan, cube, k, lam, eps, n_iter, mask, reps)
        plan.close()
        results.append((ms, t))
        if verbose:
            print(f"  pixel_rows={pr:5d} stat_rows={sr:5d} persistent={pq}: {ms:.3f} ms")
    if results_out is not None:
        results_out.extend(results)
    ms, best = min(results, key=lambda r: r[0])
    if use_cache:
        cache[key] = {"tuning": best, "ms": ms,
                      "candidates": [{"tuning": t, "ms": m} for m, t in results]}
        save_cache(cache)
    return dict(best)
