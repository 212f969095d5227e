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
