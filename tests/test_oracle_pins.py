"""The FP64 oracle against what the paper and the mathematics fix.

Also checks that the pins have teeth: plausible mistakes planted in copies
of the oracle (on the CPU) must each fail at least one pin."""
import inspect
import types

import numpy as np
import pytest

import oracle
from oracle import mf_oracle
import oracle_pins as P
from synth import make_scene


@pytest.mark.parametrize("pin", P.PINS, ids=lambda f: f.__name__)
def test_pin(pin):
    pin(mf_oracle)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_plume_recovery(seed):
    sc = make_scene(512, 16, 72, n_plumes=1, plume_sigma=(3.0, 3.0),
                    plume_peak=(2000.0, 2000.0), seed=seed)
    P.pin_plume_recovery(mf_oracle, sc)


def test_not_spd_and_small_partition():
    X, k, _ = P.tiny_partition(N=6, B=6)
    with pytest.raises(oracle.NotSPD):
        oracle.retrieve_partition(X, k, n_iter=2)
    rows, cols, B = 20, 2, 6
    X, k, _ = P.tiny_partition(N=rows * cols, B=B, seed=3)
    cube = X.reshape(rows, cols, B).copy()
    mask = np.zeros((rows, cols), np.uint8)
    mask[:16, 1] = 1                   # column 1 keeps 4 <= B pixels
    a, st = oracle.retrieve(cube, k, 1e-3, 1e-9, 2, mask=mask)
    assert st[0] == 0 and st[1] == oracle.STATUS_NOT_SPD
    assert np.isnan(a[16:, 1]).all() and (a[:16, 1] == 0).all()
    assert np.isfinite(a[:, 0]).all()


def test_band_window():
    rows, cols, B = 30, 2, 6
    X, k, _ = P.tiny_partition(N=rows * cols, B=B, seed=8)
    cube = X.reshape(rows, cols, B)
    pad = np.concatenate([np.full((rows, cols, 3), np.nan), cube, np.ones((rows, cols, 2))], -1)
    a, _ = oracle.retrieve(cube, k, 1e-3, 1e-9, 3)
    b, _ = oracle.retrieve(pad, k, 1e-3, 1e-9, 3, band_lo=3, band_hi=3 + B)
    np.testing.assert_array_equal(a, b)


# --------------------------------------------------------------- mutations
MUTATIONS = {
    "beta_without_albedo": ("beta = np.where(rpos, r * alpha, 0.0)", "beta = alpha.copy()"),
    "mean_uses_new_target": (
        "mu_new = mean_vector(X - beta[:, None] * t[None, :])",
        "mu_new = mean_vector(X - beta[:, None] * (mean_vector(X) * s)[None, :])"),
    "residual_uses_old_target": (
        "D = X - beta[:, None] * t_new[None, :] - mu_new",
        "D = X - beta[:, None] * t[None, :] - mu_new"),
    "residual_drops_mean": (
        "D = X - beta[:, None] * t_new[None, :] - mu_new",
        "D = X - beta[:, None] * t_new[None, :] - mean_vector(X)"),
    "no_alpha0_clamp": ("alpha = np.maximum(alpha, 0.0)                    # R3",
                        "alpha = alpha"),
    "penalty_sign": ("pre = np.where(rpos, (p - pen)", "pre = np.where(rpos, (p + pen)"),
    "denominator_without_r": ("(p - pen) / np.where(rpos, r * q, 1.0)",
                              "(p - pen) / np.where(rpos, q, 1.0)"),
    "init_without_r": ("alpha = np.where(rpos, p / np.where(rpos, r * q, 1.0), 0.0)",
                       "alpha = np.where(rpos, p / np.where(rpos, q, 1.0), 0.0)"),
    "albedo_uses_squared_norm_wrong": ("return (X @ mu) / (mu @ mu)",
                                       "return (X @ mu) / np.sqrt(mu @ mu)"),
    "mean_wrong_normalisation": ("return X.sum(axis=0) / X.shape[0]",
                                 "return X.sum(axis=0) / (X.shape[0] + 1)"),
    "cov_unbiased": ("return (D.T @ D) / D.shape[0]", "return (D.T @ D) / (D.shape[0] - 1)"),
    "cov_transposed_scalar": ("return (D.T @ D) / D.shape[0]",
                              "return np.diag(np.sum(D * D, axis=0)) / D.shape[0]"),
    "weights_without_eps": ("w = 1.0 / (alpha + eps) if use_sparse",
                            "w = 1.0 / (alpha + 1.0) if use_sparse"),
    "target_wrong_mean": ("t_new = target_spectrum(mu_new, s)", "t_new = target_spectrum(mu, s)"),
    "no_albedo_pen_ignored": ("if no_albedo_pen:", "if False:"),
    "mask_ignored": ("ok &= (np.asarray(mask) == 0)", "ok &= True"),
    "energy_penalty_halved": ("E[k] = float(np.sum(D.T * Z) + 2.0 * np.sum(tr[\"pen\"][k] * ra))",
                              "E[k] = float(np.sum(D.T * Z) + np.sum(tr[\"pen\"][k] * ra))"),
    "energy_initial_clamped": ("        a = tr[\"alpha\"][k]\n        ra = np.where(r > 0, r * a, 0.0)",
                               "        a = np.maximum(tr[\"alpha\"][k], 0.0)\n        ra = np.where(r > 0, r * a, 0.0)"),
    "energy_without_albedo_in_residual": ("        ra = np.where(r > 0, r * a, 0.0)\n        D = (X",
                                          "        ra = np.where(r > 0, a, 0.0)\n        D = (X"),
    # the amplification factor that widens the per-pixel parity bound
    "amplification_w_not_squared": ("kap = lam * w * w / np.where(r > 0, r * q, np.inf)",
                                    "kap = lam * w / np.where(r > 0, r * q, np.inf)"),
    "amplification_without_r": ("kap = lam * w * w / np.where(r > 0, r * q, np.inf)",
                                "kap = lam * w * w / np.where(r > 0, q, np.inf)"),
    "amplification_clamp_ignored": ("kap = np.where(tr[\"alpha\"][k] > 0, kap, 0.0)", "kap = kap"),
    "amplification_not_compounded": ("A = 1.0 + kap * A", "A = 1.0 + kap"),
    "amplification_penalty_flag_ignored": (
        "        if flags & PENALTY_NO_ALBEDO:\n            kap = kap /",
        "        if False:\n            kap = kap /"),
}


def _mutant(old, new):
    src = inspect.getsource(mf_oracle)
    assert src.count(old) >= 1, old
    src = src.replace(old, new)
    mod = types.ModuleType("mutant")
    exec(compile(src, "mutant", "exec"), mod.__dict__)
    return mod


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_pins_catch_mutation(name):
    old, new = MUTATIONS[name]
    mod = _mutant(old, new)
    failures = []
    for pin in P.PINS:
        try:
            with np.errstate(all="ignore"):
                pin(mod)
        except Exception as e:  # AssertionError, or a crash of the mutant
            failures.append(pin.__name__)
    assert failures, f"mutation {name} survived every pin"


def test_golden_regression():
    """The oracle still reproduces the values its committed script stored."""
    import json
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", "tiny_oracle.json")) as f:
        g = json.load(f)
    X, s = np.array(g["X"]), np.array(g["s"])
    for case in g["cases"]:
        a = oracle.retrieve_partition(X, s, lam=case["lam"], eps=case["eps"],
                                      n_iter=case["n_iter"], flags=case["flags"])
        np.testing.assert_allclose(a, case["alpha"], rtol=1e-12, atol=1e-9)
