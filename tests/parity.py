"""Helpers shared by the GPU parity tests: oracle runs and the alpha metric."""
from __future__ import annotations

import math

import numpy as np

# FP32 path against the FP64 oracle: normwise relative error bound on alpha
TOL_FP32 = 1e-4
# ceiling on the amplification factor that may widen one pixel's bound: a
# pixel amplified more than this is still checked, at this factor
AMP_CAP = 1e3
# pixels with A_i > AMP_STRONG are the strongly amplified ones: at most
# AMP_FRAC of the valid pixels may be (a property of the scene and the
# iteration count, checked so that the widening cannot cover a large share)
AMP_STRONG = 10.0
AMP_FRAC = 1e-2
# of the other pixels (A_i <= AMP_STRONG) at most this fraction (rounded up)
# may use the widening, i.e. miss the plain bound tol * max|ref|
WIDEN_FRAC = 1e-4


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


def alpha_report(got, ref, valid, amp, tol=TOL_FP32):
    """Every figure of the parity bar (see ``check_alpha``) without asserting:
    e_inf, e_2, e_sc (the error scaled by the capped amplification factor),
    n_valid, n_amp (pixels with A_i > AMP_STRONG), max_amp, n_widened (pixels
    with A_i <= AMP_STRONG beyond the plain bound tol * max|ref|) and
    n_widen_max (how many of those may be)."""
    g = np.asarray(got, dtype=np.float64)[valid]
    r = np.asarray(ref, dtype=np.float64)[valid]
    a = np.asarray(amp, dtype=np.float64)[valid]
    e_inf, e_2 = alpha_errors(got, ref, valid)
    scale = max(np.abs(r).max(), 1e-30) if r.size else 1.0
    d = np.abs(g - r)
    e_sc = float((d / (scale * np.minimum(a, AMP_CAP))).max()) if r.size else 0.0
    return {"e_inf": e_inf, "e_2": e_2, "e_sc": e_sc, "n_valid": int(r.size),
            "n_amp": int((a > AMP_STRONG).sum()), "max_amp": float(a.max()) if r.size else 1.0,
            "n_widened": int(((d > tol * scale) & (a <= AMP_STRONG)).sum()),
            "n_widen_max": int(math.ceil(WIDEN_FRAC * r.size))}


def check_alpha(got, ref, valid, amp, tol=TOL_FP32):
    """The parity bar for float32 paths:
    * e_2 (normwise relative, all valid pixels) <= tol;
    * every pixel: |got - ref| <= tol * max|ref| * min(A_i, AMP_CAP), where
      A_i >= 1 is the oracle's amplification factor of the reweighting map at
      that pixel (``oracle.amplification``): the derivative of the shrinkage
      step with respect to the previous estimate is lam w^2 / (r q), so where
      the previous estimate was tiny and positive any rounding is magnified,
      in every precision.  A_i is capped at AMP_CAP, so no pixel goes
      unchecked;
    * at most AMP_FRAC of the pixels may be strongly amplified (A_i >
      AMP_STRONG), and of the others at most ceil(WIDEN_FRAC * n_valid) may
      use the widening, i.e. exceed the plain bound tol * max|ref|: an error
      spread over many mildly amplified pixels fails.
    Returns the dict of ``alpha_report``."""
    rep = alpha_report(got, ref, valid, amp, tol)
    info = (f"(e_inf {rep['e_inf']:.3e}, e_2 {rep['e_2']:.3e}, {rep['n_amp']} of "
            f"{rep['n_valid']} pixels with A > {AMP_STRONG:g}, max A {rep['max_amp']:.3g}, "
            f"{rep['n_widened']} others beyond the plain bound, at most {rep['n_widen_max']})")
    assert rep["e_2"] <= tol, f"e_2 {rep['e_2']:.3e} > {tol} {info}"
    assert rep["e_sc"] <= tol, f"amplification-scaled e_inf {rep['e_sc']:.3e} > {tol} {info}"
    assert rep["n_amp"] <= AMP_FRAC * rep["n_valid"], f"too many amplified pixels {info}"
    assert rep["n_widened"] <= rep["n_widen_max"], f"too many widened pixels {info}"
    return rep
