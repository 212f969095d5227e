"""The seeded scene generator (synth/): the two Beer-Lambert forward models.

The generator only draws inputs; these tests pin that the exponential model
differs from the linearised one by exactly the transmittance ratio, pixel by
pixel, on the same random draws (Sec. II-A: L = L0 exp(-alpha s); Eq. (1) keeps
its first-order expansion, with k = -s here)."""
import numpy as np
import pytest

from synth import make_scene


def _pair(**kw):
    lin = make_scene(forward_model="linear", **kw)
    ex = make_scene(forward_model="exp", **kw)
    return lin, ex


def test_exp_model_is_transmittance_ratio_of_linear():
    lin, ex = _pair(rows=64, cols=5, bands=72, n_plumes=2, plume_sigma=(3.0, 6.0),
                    plume_peak=(1000.0, 4000.0), seed=11)
    ak = lin.alpha_true[:, :, None] * lin.k[None, None, :]
    want = np.exp(ak) / (1.0 + ak)
    got = ex.cube.numpy().astype(np.float64) / lin.cube.numpy().astype(np.float64)
    np.testing.assert_allclose(got, want, rtol=5e-7)
    # outside the plumes the two models coincide
    clear = lin.alpha_true == 0
    assert clear.any()
    np.testing.assert_array_equal(ex.cube.numpy()[clear], lin.cube.numpy()[clear])


def test_exp_model_absorbs_more_weakly_than_the_linearisation():
    """exp(x) >= 1 + x for every x: with k <= 0 the exponential model keeps
    more radiance than its first-order expansion wherever a plume is."""
    lin, ex = _pair(rows=48, cols=4, bands=72, n_plumes=1, plume_sigma=(4.0, 4.0),
                    plume_peak=(5000.0, 5000.0), seed=3)
    plume = lin.alpha_true > 0
    assert np.all(ex.cube.numpy()[plume] >= lin.cube.numpy()[plume] * (1 - 1e-7))


def test_unknown_forward_model_rejected():
    with pytest.raises(ValueError):
        make_scene(rows=8, cols=2, bands=8, forward_model="quadratic")
