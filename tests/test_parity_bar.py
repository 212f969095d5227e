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
