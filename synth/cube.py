"""Seeded synthetic radiance cubes shaped like AVIRIS-NG flightlines.

This module only draws inputs: it holds none of the retrieval's arithmetic.
Both the CUDA path and the FP64 oracle consume what it produces, so that
neither side ever supplies the other's inputs.

Generative model (linearised Beer-Lambert forward model, Eq. (1) of Foote et
al. 2020, with the scene structure of Sec. II-F/II-G and Sec. III):

  x_i = a_i (mu_c + z_i) (.) (1 + alpha_i k)         (forward_model="linear")
  x_i = a_i (mu_c + z_i) (.) exp(alpha_i k)           (forward_model="exp": the
        Beer-Lambert law itself, Sec. II-A, before the first-order expansion
        that Eq. (1) makes; k <= 0, so exp(alpha k) is the transmittance)
  z_i ~ N(0, C_bg),  C_bg = U U^T + diag(sigma^2),  sigma_b = mu_b / SNR_b
  a_i ~ lognormal(0, albedo_sigma)           per-pixel albedo
  k   = -sum_j A_j exp(-(wl - c_j)^2 / 2 s_j^2), min_b k_b = -1e-4 (ppm m)^-1
  alpha: Gaussian plume blobs A exp(-d^2 / 2 sigma^2), truncated at 0.05 A

* 72 band centres uniform over 2122-2488 nm (about 5 nm spacing, Sec. II-F);
* mu_bg is a smooth positive spectrum scaled to [1, 10] (low-order cosines);
  each detector column gets its own gain (pushbroom detector response,
  Sec. II-E), so each column has its own background;
* U is 8 smooth cosine modes with geometrically decaying scales, scaled so
  that cond(C_bg) equals ``cond``;
* the mask is Bernoulli(mask_frac) per pixel, or a per-column fraction.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import torch


def wavelengths(bands: int = 72, lo: float = 2122.0, hi: float = 2488.0) -> np.ndarray:
    return np.linspace(lo, hi, bands)


def absorption_spectrum(wl: np.ndarray, n_lines: int = 12, peak: float = 1e-4,
                        seed: int = 0) -> np.ndarray:
    """Unit absorption spectrum k (float64, negative, min = -peak)."""
    rng = np.random.default_rng(seed + 1009)
    c = rng.uniform(wl[0], wl[-1], n_lines)
    s = rng.uniform(3.0, 12.0, n_lines)
    A = rng.uniform(0.2, 1.0, n_lines)
    k = -(A[None, :] * np.exp(-((wl[:, None] - c[None, :]) ** 2) / (2 * s[None, :] ** 2))).sum(1)
    return k * (peak / np.abs(k.min()))


def background_model(wl: np.ndarray, rank: int = 8, cond: float = 1e4,
                     snr=(100.0, 500.0), seed: int = 0):
    """(mu_bg, U, sigma): smooth mean in [1, 10], low-rank factor, noise std."""
    rng = np.random.default_rng(seed + 2003)
    B = wl.shape[0]
    u = (wl - wl[0]) / (wl[-1] - wl[0])
    coef = rng.normal(0.0, 1.0, 5) / (1.0 + np.arange(5))
    base = sum(cf * np.cos(math.pi * m * u) for m, cf in enumerate(coef))
    mu = 1.0 + 9.0 * (base - base.min()) / (base.max() - base.min() + 1e-12)
    snr_b = rng.uniform(snr[0], snr[1], B)
    sigma = mu / snr_b
    modes = np.stack([np.cos(math.pi * (m + 1) * u + rng.uniform(0, math.pi))
                      for m in range(rank)], axis=1)
    scales = 0.5 ** np.arange(rank)
    U0 = modes * scales[None, :] * (1.0 + 0.2 * rng.normal(size=(1, rank)))

    def cond_of(f):
        Cb = f * f * (U0 @ U0.T) + np.diag(sigma ** 2)
        ev = np.linalg.eigvalsh(Cb)
        return ev[-1] / ev[0]

    lo_f, hi_f = 0.0, 1.0
    while cond_of(hi_f) < cond:
        hi_f *= 2.0
        if hi_f > 1e8:
            break
    for _ in range(80):
        mid = 0.5 * (lo_f + hi_f)
        if cond_of(mid) < cond:
            lo_f = mid
        else:
            hi_f = mid
    return mu, U0 * hi_f, sigma


def plume_map(rows: int, cols: int, n_plumes: int, sigma_range, peak_range,
              rng: np.random.Generator) -> np.ndarray:
    """Sum of truncated Gaussian blobs (float64, ppm m)."""
    alpha = np.zeros((rows, cols))
    for _ in range(n_plumes):
        r0 = rng.uniform(0, rows)
        c0 = rng.uniform(0, cols)
        sg = rng.uniform(*sigma_range)
        A = rng.uniform(*peak_range)
        rad = sg * math.sqrt(2.0 * math.log(20.0))
        ra, rb = max(0, int(r0 - rad) - 1), min(rows, int(r0 + rad) + 2)
        ca, cb = max(0, int(c0 - rad) - 1), min(cols, int(c0 + rad) + 2)
        rr = np.arange(ra, rb)[:, None] + 0.5
        cc = np.arange(ca, cb)[None, :] + 0.5
        blob = A * np.exp(-((rr - r0) ** 2 + (cc - c0) ** 2) / (2 * sg * sg))
        blob[blob < 0.05 * A] = 0.0
        alpha[ra:rb, ca:cb] += blob
    return alpha


@dataclass
class Scene:
    cube: torch.Tensor          # (rows, cols, bands) float32, BIP
    k: np.ndarray               # (bands,) float64 unit absorption spectrum
    mask: torch.Tensor | None   # (rows, cols) uint8, nonzero = excluded
    alpha_true: np.ndarray      # (rows, cols) float64
    albedo: np.ndarray | None = None
    mu_bg: np.ndarray | None = None
    C_bg: np.ndarray | None = None
    wl: np.ndarray | None = None
    meta: dict = field(default_factory=dict)


def make_scene(rows: int, cols: int, bands: int = 72, *, n_plumes: int = 1,
               plume_sigma=(3.0, 3.0), plume_peak=(2000.0, 2000.0), mask_frac=0.0,
               mask_col_frac=None, cond: float = 1e4, snr=(100.0, 500.0),
               albedo_sigma: float = 0.2, seed: int = 0, device="cpu",
               nan_masked: bool = False, keep_truth: bool = True,
               forward_model: str = "linear", out=None, mask_out=None) -> Scene:
    """Draw one scene.  ``device`` is where the cube is generated (torch
    Philox on CUDA, torch CPU generator otherwise).  ``forward_model``:
    "linear" (first-order Beer-Lambert, the model the filter assumes) or
    "exp" (the unlinearised Beer-Lambert transmittance).  ``out`` /
    ``mask_out``: optional contiguous (rows, cols, bands) float32 and
    (rows, cols) uint8 tensors on ``device`` to draw into (for example row
    slices of one stacked batch), instead of new ones."""
    if forward_model not in ("linear", "exp"):
        raise ValueError("forward_model must be 'linear' or 'exp'")
    wl = wavelengths(bands)
    k = absorption_spectrum(wl, seed=seed)
    mu_bg, U, sigma = background_model(wl, cond=cond, snr=snr, seed=seed)
    rng = np.random.default_rng(seed)
    alpha = plume_map(rows, cols, n_plumes, plume_sigma, plume_peak, rng) if n_plumes else \
        np.zeros((rows, cols))
    gain = 1.0 + 0.01 * rng.normal(size=cols)

    dev = torch.device(device)
    g = torch.Generator(device=dev)
    g.manual_seed(int(seed) * 7919 + 17)
    f32 = torch.float32
    Ut = torch.as_tensor(U, dtype=f32, device=dev)
    sg = torch.as_tensor(sigma, dtype=f32, device=dev)
    mu_t = torch.as_tensor(mu_bg, dtype=f32, device=dev)
    k_t = torch.as_tensor(k, dtype=f32, device=dev)
    gain_t = torch.as_tensor(gain, dtype=f32, device=dev)
    if out is not None:
        assert tuple(out.shape) == (rows, cols, bands) and out.dtype == f32 and out.is_contiguous()
        cube = out
    else:
        cube = torch.empty((rows, cols, bands), dtype=f32, device=dev)
    albedo = torch.empty((rows, cols), dtype=f32, device=dev)
    chunk = max(1, (1 << 24) // max(1, cols * bands))
    alpha_t = torch.as_tensor(alpha, dtype=f32, device=dev)
    for r0 in range(0, rows, chunk):
        r1 = min(rows, r0 + chunk)
        n = r1 - r0
        eta = torch.randn((n, cols, U.shape[1]), generator=g, device=dev, dtype=f32)
        xi = torch.randn((n, cols, bands), generator=g, device=dev, dtype=f32)
        z = eta @ Ut.T + xi * sg
        a = torch.exp(albedo_sigma * torch.randn((n, cols), generator=g, device=dev, dtype=f32))
        albedo[r0:r1] = a
        bg = mu_t[None, None, :] * gain_t[None, :, None] + z
        ak = alpha_t[r0:r1, :, None] * k_t[None, None, :]
        trans = torch.exp(ak) if forward_model == "exp" else 1.0 + ak
        cube[r0:r1] = a[:, :, None] * bg * trans
    mask = None
    if mask_frac or mask_col_frac is not None:
        if mask_col_frac is not None:
            frac = torch.as_tensor(np.asarray(mask_col_frac, dtype=np.float32), device=dev)
            u = torch.rand((rows, cols), generator=g, device=dev)
            mask = (u < frac[None, :]).to(torch.uint8)
        else:
            u = torch.rand((rows, cols), generator=g, device=dev)
            mask = (u < mask_frac).to(torch.uint8)
        if nan_masked:
            cube[mask.bool()] = float("nan")
        if mask_out is not None:
            mask_out.copy_(mask)
            mask = mask_out
    C_bg = U @ U.T + np.diag(sigma ** 2)
    return Scene(cube=cube, k=k, mask=mask, alpha_true=alpha if keep_truth else None,
                 albedo=albedo.cpu().numpy() if keep_truth and rows * cols <= (1 << 24) else None,
                 mu_bg=mu_bg, C_bg=C_bg, wl=wl,
                 meta=dict(rows=rows, cols=cols, bands=bands, seed=seed, cond=cond,
                           forward_model=forward_model))


# Named workloads (shapes of the five configurations the benchmarks and the
# parity tests use).  lam is the multiplier on the paper's weight, eps the
# reweighting constant of Eq. (5).
WORKLOADS = {
    "plain-512x16x72": dict(rows=512, cols=16, bands=72, n_plumes=1, plume_sigma=(3.0, 3.0),
                            plume_peak=(2000.0, 2000.0), mask_frac=0.0, lam=1e-3, eps=1e-9,
                            n_iter=10),
    "flightline-4000x598x72": dict(rows=4000, cols=598, bands=72, n_plumes=20,
                                   plume_sigma=(3.0, 15.0), plume_peak=(500.0, 5000.0),
                                   mask_frac=0.05, lam=1e-3, eps=1e-9, n_iter=10),
    "precision-20000x598x72": dict(rows=20000, cols=598, bands=72, n_plumes=20,
                                   plume_sigma=(3.0, 15.0), plume_peak=(500.0, 5000.0),
                                   mask_frac=0.05, lam=1e-3, eps=1e-9, n_iter=10, cond=1e7,
                                   snr=(100.0, 500.0)),
    # the flightline with the unlinearised (exponential) Beer-Lambert forward model
    "flightline-exp-4000x598x72": dict(rows=4000, cols=598, bands=72, n_plumes=20,
                                       plume_sigma=(3.0, 15.0), plume_peak=(500.0, 5000.0),
                                       mask_frac=0.05, lam=1e-3, eps=1e-9, n_iter=10,
                                       forward_model="exp"),
    "diff-8000x598x72": dict(rows=8000, cols=598, bands=72, n_plumes=20,
                             plume_sigma=(3.0, 15.0), plume_peak=(500.0, 5000.0),
                             mask_frac=0.05, lam=1e-3, eps=1e-9, n_iter=10),
}


def workload_scene(name: str, seed: int = 0, device="cpu", **over) -> tuple[Scene, dict]:
    """Scene plus the retrieval parameters (lam, eps, n_iter) of a named workload."""
    w = dict(WORKLOADS[name])
    w.update(over)
    params = {k: w.pop(k) for k in ("lam", "eps", "n_iter")}
    return make_scene(seed=seed, device=device, **w), params


def batched_lines(n_lines: int = 64, cols: int = 598, bands: int = 72,
                  rows_range=(2000, 30000), seed: int = 0):
    """Per-flightline shapes and parameters of the batched workload: rows
    uniform in ``rows_range``, per-column masked fraction U(0, 0.3), n_iter
    uniform in 5..20, lam log-uniform in [1e-4, 1e-2]."""
    rng = np.random.default_rng(seed + 4242)
    out = []
    for i in range(n_lines):
        out.append(dict(rows=int(rng.integers(rows_range[0], rows_range[1] + 1)), cols=cols,
                        bands=bands, mask_col_frac=rng.uniform(0.0, 0.3, cols),
                        n_iter=int(rng.integers(5, 21)),
                        lam=float(10 ** rng.uniform(-4, -2)), eps=1e-9, seed=seed * 1000 + i))
    return out
