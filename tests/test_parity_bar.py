"""The alpha parity bar itself (tests/parity.py), on the CPU: it must reject
an error spread over many moderately amplified pixels, and it must still
check a pixel whose amplification factor is enormous."""
import numpy as np
import pytest

from parity import AMP_CAP, AMP_FRAC, TOL_FP32, alpha_report, check_alpha


def _case(n=20000, seed=0):
    rng = np.random.default_rng(seed)
    ref = np.where(rng.random(n) < 0.1, rng.uniform(100.0, 3000.0, n), 0.0)
    valid = np.ones(n, bool)
    return ref, valid


def test_clean_result_passes():
    ref, valid = _case()
    got = ref * (1 + 1e-7)
    rep = check_alpha(got, ref, valid, np.ones_like(ref))
    assert rep["n_widened"] == 0 and rep["max_amp"] == 1.0


def test_error_spread_over_amplified_pixels_fails():
    """Every pixel mildly amplified (5-fold), 0.5% of them wrong by twice the
    plain bound: each pixel is inside its widened bound and e_2 stays below
    the bar, but far more than 1e-4 of the pixels use the widening."""
    ref, valid = _case()
    amp = np.full_like(ref, 5.0)
    scale = np.abs(ref).max()
    got = ref.copy()
    idx = np.arange(0, ref.size, 200)           # 0.5% of the pixels, each wrong by
    got[idx] += 2 * TOL_FP32 * scale             # twice the plain bound
    rep = alpha_report(got, ref, valid, amp)
    assert rep["e_2"] < TOL_FP32 and rep["e_sc"] <= TOL_FP32
    with pytest.raises(AssertionError, match="widened"):
        check_alpha(got, ref, valid, amp)


def test_huge_amplification_is_capped():
    """A pixel with A = 1e12 is checked at AMP_CAP, not left unchecked."""
    n = 4_000_000                               # large enough that e_2 hides one pixel
    ref = np.full(n, 3000.0)
    valid = np.ones(n, bool)
    amp = np.ones_like(ref)
    amp[7] = 1e12
    scale = 3000.0
    got = ref.copy()
    got[7] += 1.5 * AMP_CAP * TOL_FP32 * scale
    rep = alpha_report(got, ref, valid, amp)
    assert rep["e_2"] < TOL_FP32
    with pytest.raises(AssertionError, match="amplification-scaled"):
        check_alpha(got, ref, valid, amp)
    got[7] = ref[7] + 0.5 * AMP_CAP * TOL_FP32 * scale
    rep = check_alpha(got, ref, valid, amp)
    assert rep["n_widened"] == 0 and rep["n_amp"] == 1 and rep["n_widen_max"] == 400


def test_strong_amplification_of_many_pixels_fails():
    """A widening that would cover more than AMP_FRAC of the pixels (each
    amplified 50-fold) is refused even when every error is within it."""
    ref, valid = _case()
    amp = np.ones_like(ref)
    amp[: int(2 * AMP_FRAC * ref.size)] = 50.0
    with pytest.raises(AssertionError, match="amplified pixels"):
        check_alpha(ref.copy(), ref, valid, amp)


def test_zero_flips_are_counted_and_capped():
    """A near-threshold pixel where one side clamped to 0 and the other did
    not is left out of e_2 and the per-pixel bound, but counted: at most
    ceil(1e-4 n) of them."""
    ref, valid = _case(n=20000)
    got = ref.copy()
    near = np.zeros_like(valid)
    z = np.nonzero(ref == 0)[0][:3]
    got[z] = 500.0                               # three pixels that stayed positive
    near[z] = True
    amp = np.ones_like(ref)
    with pytest.raises(AssertionError):
        check_alpha(got, ref, valid, amp)        # without the marking: a plain failure
    with pytest.raises(AssertionError, match="zero-flips"):
        check_alpha(got, ref, valid, amp, near=near)   # 3 > ceil(2)
    got[z[2]] = 0.0
    rep = check_alpha(got, ref, valid, amp, near=near)
    assert rep["n_flips"] == 2 and rep["n_near"] == 3 and rep["e_2"] == 0.0


def test_near_threshold_marks_the_flips_of_float32_sized_perturbations():
    """The oracle on inputs perturbed by 1e-7 relative (float32 rounding)
    clamps some pixels on the other side of zero than on the exact inputs;
    every such zero-flip must be among the pixels ``near_threshold`` marks."""
    import oracle
    from parity import f32, near_threshold
    from synth import workload_scene
    sc, prm = workload_scene("flightline-4000x598x72", seed=3, cols=40)
    cube = sc.cube.numpy().astype(np.float64)
    valid = oracle.valid_pixels(cube, sc.mask.numpy())
    flips = covered = 0
    for c in range(cube.shape[1]):
        X = cube[:, c][valid[:, c]]
        Xp = X * (1 + 1e-7 * np.random.default_rng(c).standard_normal(X.shape))
        a = oracle.retrieve_partition(X, f32(sc.k), prm["lam"], prm["eps"], 10)
        b = oracle.retrieve_partition(Xp, f32(sc.k), prm["lam"], prm["eps"], 10)
        near = near_threshold(X, f32(sc.k), prm["lam"], prm["eps"], 10)
        flip = ((a == 0) | (b == 0)) & (np.abs(a - b) > 1e-6 * np.abs(a).max())
        flips += int(flip.sum())
        covered += int((flip & near).sum())
    assert flips >= 1 and covered == flips, (flips, covered)
