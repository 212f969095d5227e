"""FP64 oracle of the gradient of the retrieval (the differentiation form).

TEST INFRASTRUCTURE ONLY (same rule as ``mf_oracle``): only the test suite,
``__graft_entry__.smoke()`` and ``bench.py`` may import it.

An independent restatement of Fig. 1 (Algorithm AlbedoReWeightL1Filter) in
float64 torch operations on the CPU, so that reverse-mode automatic
differentiation gives the vector-Jacobian product of the unrolled iterations
with respect to the radiance cube, the unit absorption spectrum s and the
weight multiplier lambda.  Steps, per partition and in the paper's order:
initial mean and covariance, albedo factor r_i (Eq. (7)), target t = mu (.) s
(Eq. (9)), initial estimate (Eq. (3) divided by r_i), then for every
iteration the weights (Eq. (5)), the mean with the enhancement removed
(Eq. (10)), the covariance of d_i (Eq. (11)) and the non-negative shrinkage.
Linear systems go through a Cholesky factor (torch.linalg.cholesky and
torch.cholesky_solve).  The clamp max(., 0) is torch.relu, whose derivative
at exactly 0 is 0 (the subgradient convention at the kink).  The readings are
those of ``mf_oracle`` (R1-R10); masked and non-finite pixels are excluded and
get zero gradient.
"""
from __future__ import annotations

import numpy as np
import torch

from .mf_oracle import ALBEDO, PENALTY_NO_ALBEDO, SPARSE, partitions, valid_pixels


def retrieve_partition_t(X: torch.Tensor, s: torch.Tensor, lam: torch.Tensor, eps: float,
                         n_iter: int, flags: int = ALBEDO | SPARSE) -> torch.Tensor:
    """alpha^{n_iter} (N,) of one partition, differentiable in X (N, B), s (B,)
    and lam (scalar tensor).  Assumes N > B, SPD covariances and r_i > 0."""
    N, B = X.shape
    use_albedo = bool(flags & ALBEDO)
    use_sparse = bool(flags & SPARSE)
    no_albedo_pen = bool(flags & PENALTY_NO_ALBEDO)

    def solve(C, t):
        L = torch.linalg.cholesky(C)
        return torch.cholesky_solve(t[:, None], L)[:, 0]

    mu = X.mean(0)
    D = X - mu
    C = D.T @ D / N
    r = (X @ mu) / (mu @ mu) if use_albedo else torch.ones(N, dtype=X.dtype)
    t = mu * s
    v = solve(C, t)
    q = t @ v
    alpha = ((X - mu) @ v) / (r * q)
    if n_iter == 0:
        return alpha
    alpha = torch.relu(alpha)
    for _ in range(n_iter):
        w = 1.0 / (alpha + eps) if use_sparse else torch.zeros(N, dtype=X.dtype)
        beta = r * alpha
        mu_k = (X - beta[:, None] * t[None, :]).mean(0)
        t_k = mu_k * s
        D = X - beta[:, None] * t_k[None, :] - mu_k
        C = D.T @ D / N
        v = solve(C, t_k)
        q = t_k @ v
        p = (X - mu_k) @ v
        pen = lam * w
        if no_albedo_pen:
            pen = pen / r
        alpha = torch.relu((p - pen) / (r * q))
        t = t_k
    return alpha


def vjp(cube, s, lam, eps, n_iter, grad_alpha, mask=None, flags=ALBEDO | SPARSE,
        col_group=1):
    """Gradient of sum(grad_alpha * alpha(cube, s, lam)) over every partition.

    cube (rows, cols, B) float, s (B,), grad_alpha (rows, cols).  Returns
    (grad_cube (rows, cols, B), grad_s (B,), grad_lam) as float64 numpy;
    excluded pixels have zero gradient."""
    cube = np.asarray(cube, dtype=np.float64)
    rows, cols, B = cube.shape
    ok = valid_pixels(cube, mask)
    s_t = torch.tensor(np.asarray(s, dtype=np.float64), requires_grad=True)
    lam_t = torch.tensor(float(lam), dtype=torch.float64, requires_grad=True)
    gcube = np.zeros_like(cube)
    total = torch.zeros((), dtype=torch.float64)
    leaves = []
    for c0, c1 in partitions(cols, col_group):
        okp = ok[:, c0:c1]
        X = torch.tensor(cube[:, c0:c1][okp], requires_grad=True)
        a = retrieve_partition_t(X, s_t, lam_t, eps, n_iter, flags)
        g = torch.tensor(np.asarray(grad_alpha, dtype=np.float64)[:, c0:c1][okp])
        total = total + (g * a).sum()
        leaves.append((c0, c1, okp, X))
    total.backward()
    for c0, c1, okp, X in leaves:
        blk = np.zeros((rows, c1 - c0, B))
        blk[okp] = X.grad.numpy()
        gcube[:, c0:c1] = blk
    gl = 0.0 if lam_t.grad is None else float(lam_t.grad)  # lambda unused when n_iter = 0
    return gcube, s_t.grad.numpy().copy(), gl
