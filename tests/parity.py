"""Helpers shared by the GPU parity tests: oracle runs and the alpha metric."""
from __future__ import annotations

import math

import numpy as np

import oracle

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
# at most this fraction (rounded up) of the valid pixels may be zero-flips:
# near-threshold pixels that clamped on one side only (see near_threshold)
FLIP_FRAC = 1e-4


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


def zero_flips(got, ref, valid, amp, near, tol=TOL_FP32):
    """Near-threshold pixels (``near``) where one side is exactly 0 and the
    other differs beyond the pixel's bound: the clamp went one way on the
    GPU and the other in the oracle."""
    g = np.asarray(got, dtype=np.float64)
    r = np.asarray(ref, dtype=np.float64)
    scale = max(np.abs(r[valid]).max(), 1e-30) if valid.any() else 1.0
    bound = tol * scale * np.minimum(np.asarray(amp, np.float64), AMP_CAP)
    return valid & near & ((g == 0) | (r == 0)) & (np.abs(g - r) > bound)


def alpha_report(got, ref, valid, amp, tol=TOL_FP32, near=None, tol_pix=None):
    """Every figure of the parity bar (see ``check_alpha``) without asserting:
    e_inf, e_2, e_sc (the error scaled by the capped amplification factor),
    n_valid, n_amp (pixels with A_i > AMP_STRONG), max_amp, n_widened (pixels
    with A_i <= AMP_STRONG beyond the plain bound tol * max|ref|),
    n_widen_max (how many of those may be), n_near (near-threshold pixels),
    n_flips (zero-flips among them, left out of every other figure) and
    n_flip_max (how many may be)."""
    tol_pix = tol if tol_pix is None else tol_pix
    valid = np.asarray(valid, bool)
    n_all = int(valid.sum())
    n_near = n_flips = 0
    if near is not None:
        fl = zero_flips(got, ref, valid, amp, near, tol_pix)
        n_near, n_flips = int((valid & near).sum()), int(fl.sum())
        valid = valid & ~fl
    g = np.asarray(got, dtype=np.float64)[valid]
    r = np.asarray(ref, dtype=np.float64)[valid]
    a = np.asarray(amp, dtype=np.float64)[valid]
    e_inf, e_2 = alpha_errors(got, ref, valid)
    scale = max(np.abs(r).max(), 1e-30) if r.size else 1.0
    d = np.abs(g - r)
    e_sc = float((d / (scale * np.minimum(a, AMP_CAP))).max()) / tol_pix * tol if r.size else 0.0
    return {"e_inf": e_inf, "e_2": e_2, "e_sc": e_sc, "n_valid": int(r.size),
            "n_amp": int((a > AMP_STRONG).sum()), "max_amp": float(a.max()) if r.size else 1.0,
            "n_widened": int(((d > tol_pix * scale) & (a <= AMP_STRONG)).sum()),
            "n_widen_max": int(math.ceil(WIDEN_FRAC * r.size)),
            "n_near": n_near, "n_flips": n_flips, "n_flip_max": int(math.ceil(FLIP_FRAC * n_all))}


def near_threshold(X, s, lam, eps, n_iter, flags=oracle.ALBEDO | oracle.SPARSE, alpha_init=None,
                   tau=TOL_FP32):
    """Pixels of one partition whose clamp max(0, .) is not determined at the
    parity bar's precision: at some iteration k >= 1 the oracle's unclamped
    update |pre_i^k| is within tau * max|alpha| * max(1, kappa_i^k A_i^{k-1})
    of zero, the error the bar allows for the previous estimate (A_i^{k-1},
    as in ``oracle.amplification``) carried through the step's derivative
    kappa_i^k = lam w^2 / (r q) (the derivative on the unclamped side).  Such
    a pixel may clamp on one side and not on the other, and with the sticky
    zero of the reweighting (w = 1/eps) the two trajectories then part."""
    N = X.shape[0]
    flag = np.zeros(N, bool)
    _, tr = oracle.retrieve_partition(X, s, lam, eps, n_iter, flags, alpha_init, trace=True)
    if n_iter == 0:
        return flag
    scale = max(np.abs(tr["alpha"][-1]).max(), 1e-30)
    r = tr["r"]
    prev = np.maximum(tr["alpha"][0] if alpha_init is None else np.asarray(alpha_init, float), 0.0)
    A = np.ones(N)
    for k in range(1, n_iter + 1):
        q = tr["q"][k]
        if flags & oracle.SPARSE:
            w = 1.0 / (prev + eps)
            kap = lam * w * w / np.where(r > 0, r * q, np.inf)
            if flags & oracle.PENALTY_NO_ALBEDO:
                kap = kap / np.where(r > 0, r, np.inf)
        else:
            kap = np.zeros(N)
        flag |= np.abs(tr["pre"][k]) <= tau * scale * np.maximum(1.0, np.minimum(kap * A, AMP_CAP))
        A = 1.0 + np.where(tr["alpha"][k] > 0, kap, 0.0) * A
        prev = tr["alpha"][k]
    return flag


def retrieve_near_threshold(cube, s, lam, eps, n_iter, mask=None, band_lo=0, band_hi=None,
                            col_group=1, flags=oracle.ALBEDO | oracle.SPARSE, alpha_init=None):
    """``near_threshold`` for every valid pixel of a cube (False elsewhere)."""
    cube = np.asarray(cube)
    rows, cols, bt = cube.shape
    band_hi = bt if band_hi is None else band_hi
    win = cube[:, :, band_lo:band_hi]
    ok = oracle.valid_pixels(win, mask)
    out = np.zeros((rows, cols), bool)
    for c0, c1 in oracle.partitions(cols, col_group):
        okp = ok[:, c0:c1]
        X = win[:, c0:c1][okp].astype(np.float64)
        a0 = None if alpha_init is None else np.asarray(alpha_init)[:, c0:c1][okp]
        blk = np.zeros(okp.shape, bool)
        try:
            blk[okp] = near_threshold(X, s, lam, eps, n_iter, flags, a0)
        except oracle.NotSPD:
            pass
        out[:, c0:c1] = blk
    return out


def check_alpha(got, ref, valid, amp, tol=TOL_FP32, near=None, tol_pix=None):
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
      spread over many mildly amplified pixels fails;
    * with ``near`` (the oracle's near-threshold pixels), a zero-flip among
      them (one side exactly 0, the other beyond its bound) is left out of
      the figures above; at most ceil(FLIP_FRAC * n_valid) pixels may flip.
    ``tol_pix`` (default ``tol``) replaces tol in the per-pixel bounds, for a
    form whose stated per-pixel bound differs from its e_2 bound; e_sc is
    reported in units of tol.
    Returns the dict of ``alpha_report``."""
    rep = alpha_report(got, ref, valid, amp, tol, near, tol_pix)
    info = (f"(e_inf {rep['e_inf']:.3e}, e_2 {rep['e_2']:.3e}, {rep['n_amp']} of "
            f"{rep['n_valid']} pixels with A > {AMP_STRONG:g}, max A {rep['max_amp']:.3g}, "
            f"{rep['n_widened']} others beyond the plain bound, at most {rep['n_widen_max']}; "
            f"{rep['n_flips']} zero-flips of {rep['n_near']} near-threshold pixels, at most "
            f"{rep['n_flip_max']})")
    assert rep["e_2"] <= tol, f"e_2 {rep['e_2']:.3e} > {tol} {info}"
    assert rep["e_sc"] <= tol, f"amplification-scaled e_inf {rep['e_sc']:.3e} > {tol} {info}"
    assert rep["n_amp"] <= AMP_FRAC * rep["n_valid"], f"too many amplified pixels {info}"
    assert rep["n_widened"] <= rep["n_widen_max"], f"too many widened pixels {info}"
    assert rep["n_flips"] <= rep["n_flip_max"], f"too many zero-flips {info}"
    return rep
