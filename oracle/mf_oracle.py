"""Plain FP64 CPU oracle for the albedo-corrected, reweighted-l1 matched filter.

TEST INFRASTRUCTURE ONLY.  This module exists so that the CUDA path can be
checked against an obviously correct statement of the method.  Only the test
suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import it.  The product path (the C-ABI library and its Python binding) never
calls it and has no CPU fallback.

What it computes (Foote et al., "Fast and Accurate Retrieval of Methane
Concentration from Imaging Spectrometer Data Using Sparsity Prior", IEEE TGRS
2020):

* the classic matched filter closed form, Eq. (3), as the initial estimate;
* the albedo factor r_i of Eq. (7) and the target t = mu (.) s of Eq. (9);
* the procedure of Fig. 1 (Algorithm AlbedoReWeightL1Filter), step by step,
  in the paper's order: initial mean and covariance, albedo, initial
  enhancement, then for k = 1..N_iter the weights of Eq. (5), the mean update
  of Eq. (10), the covariance update of Eq. (11) and the non-negative
  shrinkage update (Eq. (6) with the albedo factor of Sec. II-C);
* the six variants of Table I through the ALBEDO / SPARSE switches that the
  caption of Fig. 1 describes: no sparsity sets the weights to zero, no albedo
  correction sets every r_i to one.

Every statistic is recomputed literally from its defining sum at every
iteration; no rank-update identity, no blocking, no fusion.  Linear systems
C v = t are solved with a Cholesky factorisation and two triangular solves
(numpy / scipy library primitives).

Readings taken where the paper is silent or ambiguous (each is also listed in
the design notes of the repository):

R1  C^0 is the outer-product covariance (1/N) sum (L_i - mu)(L_i - mu)^T; the
    algorithm figure prints the factors transposed (a scalar), Eq. (11) and the
    update line of Fig. 1 use the outer product.
R2  r_i uses mu^0 and is computed once (the albedo line of Fig. 1 sits inside
    the initialisation loop).
R3  alpha^0 is clamped at 0 before it feeds w^1, mu^1 and C^1 (Sec. III-D: the
    positivity constraint is applied before the mean and covariance are
    computed).  With N_iter = 0 alpha^0 is returned unclamped (the
    non-iterative rows of Table I have negative values).
R4  The shrinkage step is used exactly as printed in Fig. 1:
    alpha = max(0, (p - pen) / (r q)).  The per-pixel objective it minimises
    exactly is f(a) = d^T C^-1 d + 2 pen r a on a >= 0, with
    d = (L_i - mu^k) - r a t(mu^k) (used by ``partition_energy``).
R5  pen = lam * w_i by default (penalty r_i w_i |a| of Eq. (8) in the
    r-scaled form); flag PENALTY_NO_ALBEDO gives pen = lam * w_i / r_i.
R6  lam is a dimensionless multiplier on the paper's weight; lam = 1 is the
    procedure of Fig. 1 verbatim, lam = 0 disables sparsity.
R7  Normalisation 1/N everywhere (Fig. 1, Eqs. (10)-(11)).
R8  Masked or non-finite pixels are excluded from N, mu and C and get
    alpha = 0; a partition with N <= B, or whose covariance is not positive
    definite, fails (status NOT_SPD) and gets alpha = NaN on its valid pixels.
R9  r_i <= 0 (impossible for positive radiance): alpha_i = 0 and beta_i = 0,
    the pixel still counts in the statistics.
R10 Partitions: groups of ``col_group`` adjacent detector columns, the
    remainder forming a last smaller group (Sec. II-E).
R17 The energy tracked in Fig. 5 is the sum over the partition's valid pixels
    of the bracket of Eq. (8) in the form the shrinkage step minimises exactly
    (R4, with the penalty of R5), evaluated at each iterate with that
    iterate's mu^k, C^k, t^k and weights; iterate 0 is the unclamped initial
    estimate without a penalty.

Parity pins for every function live in ``tests/test_oracle_pins.py``.
"""
from __future__ import annotations

import numpy as np
from scipy.linalg import solve_triangular

ALBEDO = 1
SPARSE = 2
LITERAL = 4  # GPU schedule switch; the oracle is always literal
PENALTY_NO_ALBEDO = 8

STATUS_OK = 0
STATUS_NOT_SPD = 4


class NotSPD(Exception):
    pass


def partitions(cols: int, col_group: int = 1):
    """Detector partitions of Sec. II-E: groups of ``col_group`` adjacent
    columns, the remaining columns form one last smaller group (R10)."""
    if col_group < 1:
        raise ValueError("col_group must be >= 1")
    return [(c0, min(c0 + col_group, cols)) for c0 in range(0, cols, col_group)]


def mean_vector(X: np.ndarray) -> np.ndarray:
    """mu = (1/N) sum_i L_i (Fig. 1, initial mean)."""
    return X.sum(axis=0) / X.shape[0]


def covariance_about(D: np.ndarray) -> np.ndarray:
    """(1/N) sum_i d_i d_i^T for the rows d_i of D (Fig. 1 / Eq. (11), R1, R7)."""
    return (D.T @ D) / D.shape[0]


def albedo_factor(X: np.ndarray, mu: np.ndarray) -> np.ndarray:
    """r_i = L_i^T mu / mu^T mu (Eq. (7))."""
    return (X @ mu) / (mu @ mu)


def target_spectrum(mu: np.ndarray, s: np.ndarray) -> np.ndarray:
    """t(mu) = mu (.) s (Eq. (9))."""
    return mu * s


def spd_solve(C: np.ndarray, b: np.ndarray) -> np.ndarray:
    """C^-1 b through C = L L^T and two triangular solves; raises NotSPD."""
    try:
        L = np.linalg.cholesky(C)
    except np.linalg.LinAlgError as e:  # not positive definite
        raise NotSPD(str(e)) from None
    y = solve_triangular(L, b, lower=True)
    return solve_triangular(L.T, y, lower=False)


def retrieve_partition(X, s, lam=1.0, eps=1e-9, n_iter=10, flags=ALBEDO | SPARSE,
                       alpha_init=None, trace=False):
    """Fig. 1 (Algorithm AlbedoReWeightL1Filter) on one partition.

    X: (N, B) valid pixel spectra L_i over the band window, any float dtype
    (promoted to float64).  s: (B,) unit absorption spectrum.
    Returns alpha (N,) and, if ``trace``, a dict of per-iteration
    intermediates (mu, C, t, v, q, p, pen, alpha, r).
    Raises NotSPD when a covariance is not positive definite or N <= B (R8).
    """
    X = np.asarray(X, dtype=np.float64)
    s = np.asarray(s, dtype=np.float64)
    N, B = X.shape
    if N <= B:
        raise NotSPD(f"N={N} <= B={B}")
    use_albedo = bool(flags & ALBEDO)
    use_sparse = bool(flags & SPARSE)
    no_albedo_pen = bool(flags & PENALTY_NO_ALBEDO)

    # --- initialisation (Fig. 1, before the k loop)
    mu = mean_vector(X)
    C = covariance_about(X - mu)                      # R1
    r = albedo_factor(X, mu) if use_albedo else np.ones(N)   # Eq. (7), R2
    rpos = r > 0                                      # R9
    t = target_spectrum(mu, s)                        # Eq. (9)
    v = spd_solve(C, t)
    q = t @ v
    p = (X - mu) @ v
    alpha = np.where(rpos, p / np.where(rpos, r * q, 1.0), 0.0)
    tr = None
    if trace:
        tr = dict(mu=[mu], C=[C], t=[t], v=[v], q=[q], p=[p], pen=[np.zeros(N)],
                  alpha=[alpha.copy()], r=r, pre=[alpha.copy()])
    if alpha_init is not None:
        alpha = np.array(alpha_init, dtype=np.float64).copy()
    if n_iter == 0:
        return (alpha, tr) if trace else alpha
    alpha = np.maximum(alpha, 0.0)                    # R3

    for _k in range(1, n_iter + 1):
        # weights, Eq. (5); w = 0 without sparsity (Fig. 1 caption)
        w = 1.0 / (alpha + eps) if use_sparse else np.zeros(N)
        beta = np.where(rpos, r * alpha, 0.0)
        # mean of the data with the current enhancement removed, Eq. (10)
        # (Fig. 1 form, with r_i): uses t(mu^{k-1})
        mu_new = mean_vector(X - beta[:, None] * t[None, :])
        t_new = target_spectrum(mu_new, s)
        # covariance update, Eq. (11) / Fig. 1: d = L - r a t(mu^k) - mu^k
        D = X - beta[:, None] * t_new[None, :] - mu_new
        C = covariance_about(D)
        v = spd_solve(C, t_new)
        q = t_new @ v
        p = (X - mu_new) @ v
        pen = lam * w
        if no_albedo_pen:
            pen = np.where(rpos, pen / np.where(rpos, r, 1.0), 0.0)
        pre = np.where(rpos, (p - pen) / np.where(rpos, r * q, 1.0), 0.0)
        alpha = np.maximum(pre, 0.0)                  # non-negative shrinkage
        mu, t = mu_new, t_new
        if trace:
            for key, val in (("mu", mu), ("C", C), ("t", t), ("v", v), ("q", q),
                             ("p", p), ("pen", pen), ("alpha", alpha.copy()),
                             ("pre", pre)):
                tr[key].append(val)
    return (alpha, tr) if trace else alpha


def valid_pixels(cube_win: np.ndarray, mask) -> np.ndarray:
    """Pixel validity (R8): not masked and every band in the window finite."""
    ok = np.all(np.isfinite(cube_win), axis=-1)
    if mask is not None:
        ok &= (np.asarray(mask) == 0)
    return ok


def retrieve(cube, s, lam=1.0, eps=1e-9, n_iter=10, mask=None, band_lo=0, band_hi=None,
             col_group=1, flags=ALBEDO | SPARSE, alpha_init=None, columns=None):
    """Whole cube: ``cube`` is (rows, cols, bands_total) BIP; the window is
    bands [band_lo, band_hi).  Each partition (R10) is retrieved independently
    (Sec. II-E).  Returns (alpha (rows, cols) float64, status (P,) int32).

    ``columns``: optional iterable of partition indices to compute (the others
    are left as NaN with status -1); used to time bounded samples.
    """
    cube = np.asarray(cube)
    rows, cols, bt = cube.shape
    if band_hi is None:
        band_hi = bt
    win = cube[:, :, band_lo:band_hi]
    s = np.asarray(s, dtype=np.float64)
    assert s.shape == (band_hi - band_lo,)
    ok = valid_pixels(win, mask)
    parts = partitions(cols, col_group)
    alpha = np.zeros((rows, cols), dtype=np.float64)
    status = np.full(len(parts), STATUS_OK, dtype=np.int32)
    sel = range(len(parts)) if columns is None else sorted(set(columns))
    if columns is not None:
        status[:] = -1
        chosen = set(sel)
        for pi, (c0, c1) in enumerate(parts):
            if pi not in chosen:
                alpha[:, c0:c1] = np.nan
    for pi in sel:
        c0, c1 = parts[pi]
        okp = ok[:, c0:c1]
        X = win[:, c0:c1][okp].astype(np.float64)          # row-major pixel order
        a0 = None
        if alpha_init is not None:
            a0 = np.asarray(alpha_init)[:, c0:c1][okp]
        blk = np.zeros(okp.shape)
        try:
            a = retrieve_partition(X, s, lam, eps, n_iter, flags, a0)
            blk[okp] = a
            status[pi] = STATUS_OK
        except NotSPD:
            blk[okp] = np.nan
            status[pi] = STATUS_NOT_SPD
        alpha[:, c0:c1] = blk
    return alpha, status


def partition_energy(X, s, lam=1.0, eps=1e-9, n_iter=10, flags=ALBEDO | SPARSE):
    """Objective of every iterate of Fig. 1 on one partition (the energy of
    Fig. 5, Sec. III-B): E^k = sum_i f_i(alpha_i^k), k = 0..n_iter, with the
    per-pixel objective f of R4 at iterate k's mu^k, C^k, t^k and pen^k,
    summed over the partition's pixels.  Iterate 0 is the
    unclamped initial estimate with no penalty (R3: the clamp feeds the first
    reweighting, it is not part of the initial estimate).  Reading R17."""
    X = np.asarray(X, dtype=np.float64)
    _, tr = retrieve_partition(X, s, lam, eps, n_iter, flags, trace=True)
    r = tr["r"]
    E = np.empty(n_iter + 1)
    for k in range(n_iter + 1):
        a = tr["alpha"][k]
        ra = np.where(r > 0, r * a, 0.0)
        D = (X - tr["mu"][k]) - ra[:, None] * tr["t"][k][None, :]
        Z = spd_solve(tr["C"][k], D.T)                 # C^-1 d_i, column per pixel
        E[k] = float(np.sum(D.T * Z) + 2.0 * np.sum(tr["pen"][k] * ra))
    return E


def retrieve_energy(cube, s, lam=1.0, eps=1e-9, n_iter=10, mask=None, band_lo=0, band_hi=None,
                    col_group=1, flags=ALBEDO | SPARSE):
    """``partition_energy`` for every partition of a cube (R10): (P, n_iter + 1)
    float64, NaN rows for partitions that fail (R8)."""
    cube = np.asarray(cube)
    rows, cols, bt = cube.shape
    if band_hi is None:
        band_hi = bt
    win = cube[:, :, band_lo:band_hi]
    ok = valid_pixels(win, mask)
    parts = partitions(cols, col_group)
    out = np.full((len(parts), n_iter + 1), np.nan)
    for pi, (c0, c1) in enumerate(parts):
        X = win[:, c0:c1][ok[:, c0:c1]].astype(np.float64)
        try:
            out[pi] = partition_energy(X, s, lam, eps, n_iter, flags)
        except NotSPD:
            pass
    return out


def amplification(X, s, lam=1.0, eps=1e-9, n_iter=10, flags=ALBEDO | SPARSE, alpha_init=None):
    """Per-pixel growth factor of a perturbation through the reweighting
    iterations, from the derivative of the shrinkage step with respect to the
    previous estimate (Eq. (5) inside the step of Fig. 1):
        kappa_i^k = d alpha_i^k / d alpha_i^{k-1}
                  = lam w_i^2 / (r_i q^k)     (lam w_i^2 / (r_i^2 q^k) with
                                               PENALTY_NO_ALBEDO)
    where alpha_i^k > 0, and 0 where the step clamps.  A perturbation of unit
    size entering at every step grows to A_i^n with A^0 = 1,
    A^k = 1 + kappa^k A^{k-1}.  Pixels with a small positive previous
    estimate have kappa >> 1: any rounding there is magnified, in every
    precision, by this factor.  Returns A (N,)."""
    _, tr = retrieve_partition(X, s, lam, eps, n_iter, flags, alpha_init, trace=True)
    N = X.shape[0]
    A = np.ones(N)
    if n_iter == 0 or not (flags & SPARSE):
        return A
    r = tr["r"]
    prev = np.maximum(tr["alpha"][0] if alpha_init is None else np.asarray(alpha_init, float), 0.0)
    for k in range(1, n_iter + 1):
        q = tr["q"][k]
        w = 1.0 / (prev + eps)
        kap = lam * w * w / np.where(r > 0, r * q, np.inf)
        if flags & PENALTY_NO_ALBEDO:
            kap = kap / np.where(r > 0, r, np.inf)
        kap = np.where(tr["alpha"][k] > 0, kap, 0.0)
        A = 1.0 + kap * A
        prev = tr["alpha"][k]
    return A


def retrieve_amplification(cube, s, lam=1.0, eps=1e-9, n_iter=10, mask=None, band_lo=0,
                           band_hi=None, col_group=1, flags=ALBEDO | SPARSE, alpha_init=None):
    """``amplification`` for every valid pixel of a cube (1 elsewhere)."""
    cube = np.asarray(cube)
    rows, cols, bt = cube.shape
    band_hi = bt if band_hi is None else band_hi
    win = cube[:, :, band_lo:band_hi]
    ok = valid_pixels(win, mask)
    out = np.ones((rows, cols))
    for (c0, c1) in partitions(cols, col_group):
        okp = ok[:, c0:c1]
        X = win[:, c0:c1][okp].astype(np.float64)
        a0 = None if alpha_init is None else np.asarray(alpha_init)[:, c0:c1][okp]
        blk = np.ones(okp.shape)
        try:
            blk[okp] = amplification(X, s, lam, eps, n_iter, flags, a0)
        except NotSPD:
            pass
        out[:, c0:c1] = blk
    return out
