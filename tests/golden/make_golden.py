"""Writes tests/golden/tiny_oracle.json from the FP64 oracle only.

The paper prints no per-pixel worked example (its experiments use AVIRIS-NG
data that is not public), so the stored values here are the oracle's own on a
tiny seeded partition: a regression fixture that detects any later change of
the oracle's arithmetic.  Run: python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))
from oracle import mf_oracle  # noqa: E402


def tiny_input():
    rng = np.random.default_rng(20200306)
    N, B = 24, 5
    mu = np.array([4.0, 6.0, 5.0, 3.0, 2.0])
    X = mu * np.exp(0.2 * rng.normal(size=(N, 1))) + 0.05 * rng.normal(size=(N, B))
    s = np.array([-1e-4, -5e-5, -2e-4, -1e-5, -8e-5])
    X[3] *= 1.0 + 3000.0 * s
    X[7] *= 1.0 + 1500.0 * s
    return np.round(X, 6), s


def main():
    X, s = tiny_input()
    out = {"X": X.tolist(), "s": s.tolist(), "cases": []}
    for n_iter, lam, flags in ((0, 0.0, 0), (0, 0.0, 1), (1, 1e-3, 3), (3, 1e-3, 3), (3, 1.0, 3),
                               (3, 1e-3, 2), (3, 0.5, 11)):
        a = mf_oracle.retrieve_partition(X, s, lam=lam, eps=1e-9, n_iter=n_iter, flags=flags)
        out["cases"].append({"n_iter": n_iter, "lam": lam, "eps": 1e-9, "flags": flags,
                             "alpha": [float(v) for v in a]})
    with open(os.path.join(HERE, "tiny_oracle.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
