"""Pins of the FP64 gradient oracle (oracle/mf_grad.py): central finite
differences of the independent numpy oracle, Euler identities of the
method's invariances, and exclusion of masked pixels."""
import numpy as np
import pytest

import oracle
from oracle import mf_oracle
from synth import make_scene

FLAGS = oracle.ALBEDO | oracle.SPARSE


def tiny(seed=0, rows=60, cols=2, bands=8, n_plumes=1):
    sc = make_scene(rows, cols, bands, n_plumes=n_plumes, plume_sigma=(3.0, 3.0),
                    plume_peak=(3000.0, 3000.0), seed=seed)
    return sc.cube.numpy().astype(np.float64), np.asarray(sc.k, np.float64)


def loss(cube, s, lam, n_iter, g, flags=FLAGS):
    a, st = oracle.retrieve(cube, s, lam, 1e-9, n_iter, flags=flags)
    assert np.all(st == 0)
    return float((g * a).sum())


def margins(cube, s, lam, n_iter, flags=FLAGS):
    """Smallest |pre-clamp value| / max|alpha| over every iteration (FD is
    only valid away from the kink)."""
    m = np.inf
    for c in range(cube.shape[1]):
        _, tr = mf_oracle.retrieve_partition(cube[:, c], s, lam, 1e-9, n_iter, flags, trace=True)
        scale = max(np.abs(a).max() for a in tr["alpha"]) + 1e-30
        for pre in tr["pre"][1:]:
            m = min(m, np.abs(pre).min() / scale)
    return m


@pytest.mark.parametrize("n_iter,lam", [(0, 0.0), (2, 0.0), (3, 1e-3)])
def test_grad_matches_central_differences(n_iter, lam):
    cube, s = tiny(seed=1)
    rng = np.random.default_rng(3)
    g = rng.normal(size=cube.shape[:2])
    if n_iter:
        assert margins(cube, s, lam, n_iter) > 1e-6
    gc, gs, gl = oracle.grad_vjp(cube, s, lam, 1e-9, n_iter, g, flags=FLAGS)
    # s: every component
    for j in range(len(s)):
        h = 1e-5 * abs(s[j])
        sp, sm = s.copy(), s.copy()
        sp[j] += h
        sm[j] -= h
        fd = (loss(cube, sp, lam, n_iter, g) - loss(cube, sm, lam, n_iter, g)) / (2 * h)
        assert fd == pytest.approx(gs[j], rel=1e-5, abs=1e-8 * np.abs(gs).max())
    # a few radiance entries
    for (i, c, b) in [(0, 0, 0), (7, 1, 3), (31, 0, 7), (59, 1, 5)]:
        h = 1e-5 * abs(cube[i, c, b])
        cp, cm = cube.copy(), cube.copy()
        cp[i, c, b] += h
        cm[i, c, b] -= h
        fd = (loss(cp, s, lam, n_iter, g) - loss(cm, s, lam, n_iter, g)) / (2 * h)
        assert fd == pytest.approx(gc[i, c, b], rel=1e-4, abs=1e-7 * np.abs(gc).max())
    if n_iter and lam > 0:
        h = 1e-5 * lam
        fd = (loss(cube, s, lam + h, n_iter, g) - loss(cube, s, lam - h, n_iter, g)) / (2 * h)
        assert fd == pytest.approx(gl, rel=1e-5)


def test_grad_s_homogeneity_without_sparsity():
    """With lambda = 0 the estimate is homogeneous of degree -1 in s (p scales
    with s, q with s^2, and beta t is invariant), so s . dL/ds = -L."""
    cube, s = tiny(seed=2)
    g = np.random.default_rng(4).normal(size=cube.shape[:2])
    for n_iter in (0, 3):
        gc, gs, gl = oracle.grad_vjp(cube, s, 0.0, 1e-9, n_iter, g)
        L = loss(cube, s, 0.0, n_iter, g)
        assert s @ gs == pytest.approx(-L, rel=1e-9)


def test_grad_cube_scale_invariance():
    """alpha is invariant to a common radiance scale (r, p/q and the weights
    are scale-free), so sum_i x_i . dL/dx_i = 0."""
    cube, s = tiny(seed=5)
    g = np.random.default_rng(6).normal(size=cube.shape[:2])
    gc, gs, gl = oracle.grad_vjp(cube, s, 1e-3, 1e-9, 3, g)
    assert abs(float((cube * gc).sum())) <= 1e-9 * float(np.abs(cube * gc).sum())


def test_grad_masked_pixels_are_excluded():
    cube, s = tiny(seed=7, rows=70)
    mask = np.zeros(cube.shape[:2], np.uint8)
    mask[::9, 0] = 1
    g = np.random.default_rng(8).normal(size=cube.shape[:2])
    gc, gs, gl = oracle.grad_vjp(cube, s, 1e-3, 1e-9, 2, g, mask=mask)
    assert np.all(gc[mask == 1] == 0)
    cube2 = cube.copy()
    cube2[mask == 1] = np.nan
    gc2, gs2, gl2 = oracle.grad_vjp(cube2, s, 1e-3, 1e-9, 2, g, mask=mask)
    np.testing.assert_array_equal(gs, gs2)
    np.testing.assert_array_equal(gc[mask == 0], gc2[mask == 0])
