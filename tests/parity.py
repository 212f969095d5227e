"""Helpers shared by the GPU parity tests: oracle runs and the alpha metric."""
from __future__ import annotations

import numpy as np

# FP32 path against the FP64 oracle: normwise relative error bound on alpha
TOL_FP32 = 1e-4


def alpha_errors(got, ref, valid):
    """e_inf = max|got - ref| / max|ref| and e_2 = ||got - ref|| / ||ref|| over
    the valid pixels."""
    g = np.asarray(got, dtype=np.float64)[valid]
    r = np.asarray(ref, dtype=np.float64)[valid]
    scale = max(np.abs(r).max(), 1e-30)
    e_inf = float(np.abs(g - r).max() / scale) if r.size else 0.0
    e_2 = float(np.linalg.norm(g - r) / max(np.linalg.norm(r), 1e-30)) if r.size else 0.0
    return e_inf, e_2


def f32(a):
    """The values the GPU receives, as float64 for the oracle."""
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def check_alpha(got, ref, valid, amp, tol=TOL_FP32):
    """The parity bar for float32 paths:
    * e_2 (normwise relative, all valid pixels) <= tol;
    * every pixel: |got - ref| <= tol * max|ref| * A_i, where A_i >= 1 is the
      oracle's amplification factor of the reweighting map at that pixel
      (``oracle.amplification``); A_i = 1 for all but a few pixels whose
      previous estimate was tiny and positive, where any rounding is magnified
      by lam w^2 / (r q) in every precision.
    Returns (e_inf, e_2, e_inf_scaled, n_amplified)."""
    g = np.asarray(got, dtype=np.float64)[valid]
    r = np.asarray(ref, dtype=np.float64)[valid]
    a = np.asarray(amp, dtype=np.float64)[valid]
    e_inf, e_2 = alpha_errors(got, ref, valid)
    scale = max(np.abs(r).max(), 1e-30) if r.size else 1.0
    e_sc = float((np.abs(g - r) / (scale * a)).max()) if r.size else 0.0
    n_amp = int((a > 10).sum())
    assert e_2 <= tol, f"e_2 {e_2:.3e} > {tol} (e_inf {e_inf:.3e})"
    assert e_sc <= tol, f"amplification-scaled e_inf {e_sc:.3e} > {tol} (raw e_inf {e_inf:.3e}, {n_amp} pixels with A > 10)"
    return e_inf, e_2, e_sc, n_amp
