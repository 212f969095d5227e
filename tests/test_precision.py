"""The precision workload: 20000 rows x 598 columns x 72 bands, background
covariance of condition number 1e7 (SNR 100-500 per band; with the albedo
variation cond(C^0) is about 1.3e7), 10 iterations, 5% of pixels masked.

The covariance of Fig. 1 / Eq. (11) is near-collinear here: its smallest
eigenvalues sit 1e7 below the largest, and t = mu (.) s has weight in their
directions.  For each form this checks, on sampled whole partitions against
the FP64 oracle, alpha (the parity bar of tests/parity.py) and C^0: the
Frobenius error ||dC||_F / ||C||_F and the error along every eigenvector u of
the oracle's C^0, |u^T dC u| / lambda_u.

* float32 statistics (fused and literal schedules): the 1e-4 alpha bar, and
  C^0 within 1e-5 along every eigenvector (the eight-direction split of the
  statistics kernel);
* BF16-split (tensor-core) statistics: their float32 accumulation inside the
  MMA chains leaves errors of order 2^-24 x (the largest entries), i.e.
  1e-2 relative along the smallest eigenvectors at this conditioning.  The
  stated bound of this form at cond 1e7 is alpha e_2 <= 5e-2 and C^0 within
  0.2 along every eigenvector (the 1e-4 alpha bar holds at cond 1e4, tested
  elsewhere).
"""
import numpy as np
import pytest
import torch

import oracle
from parity import TOL_FP32, alpha_report, check_alpha, f32, retrieve_near_threshold
from synth import workload_scene

pytestmark = pytest.mark.gpu

ALBEDO, SPARSE, LITERAL = 1, 2, 4
FP32, BF16SPLIT = 0, 1
# stated bounds at cond(C) = 1e7
C_EIG_FP32 = 1e-5
C_FRO_FP32 = 1e-6
ALPHA_E2_BF16 = 5e-2
C_EIG_BF16 = 0.2
C_FRO_BF16 = 1e-5


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2003_02978_gb300 import build
    build.build()


@pytest.fixture(scope="module")
def scene():
    sc, prm = workload_scene("precision-20000x598x72", seed=0, device="cuda")
    cols = np.unique(np.concatenate([np.random.default_rng(5).choice(598, 6, replace=False),
                                     [0, 597]]))
    sub = sc.cube[:, cols, :].cpu().numpy()
    msk = sc.mask[:, cols].cpu().numpy()
    kk = f32(sc.k)
    ref, st = oracle.retrieve(sub.astype(np.float64), kk, prm["lam"], prm["eps"], prm["n_iter"],
                              mask=msk)
    amp = oracle.retrieve_amplification(sub.astype(np.float64), kk, prm["lam"], prm["eps"],
                                        prm["n_iter"], mask=msk)
    near = retrieve_near_threshold(sub.astype(np.float64), kk, prm["lam"], prm["eps"],
                                   prm["n_iter"], mask=msk)
    valid = oracle.valid_pixels(sub, msk)
    stats = []
    for j in range(len(cols)):
        X = sub[valid[:, j], j].astype(np.float64)
        m = oracle.mean_vector(X)
        C = oracle.covariance_about(X - m)
        ev, V = np.linalg.eigh(C)
        stats.append((m, C, ev, V))
    yield dict(sc=sc, prm=prm, cols=cols, ref=ref, st=st, amp=amp, near=near, valid=valid,
               stats=stats)
    del sc
    torch.cuda.empty_cache()


def run_form(scene, flags, precision):
    import paper_2003_02978_gb300 as mfg
    sc, prm, cols = scene["sc"], scene["prm"], scene["cols"]
    plan = mfg.Plan(20000, 598, 72, flags=flags, precision=precision)
    a = plan.retrieve(sc.cube, sc.k, prm["lam"], prm["eps"], prm["n_iter"], mask=sc.mask)
    torch.cuda.synchronize()
    status = plan.status()
    mu, cov = (t[cols].cpu().numpy() for t in plan.background())
    plan.close()
    got = a[:, cols].cpu().numpy()
    assert np.all(status == 0)
    np.testing.assert_array_equal(scene["st"], 0)
    assert np.all(got[~scene["valid"]] == 0)
    c_fro, c_eig = [], []
    for j, (m, C, ev, V) in enumerate(scene["stats"]):
        dC = cov[j] - C
        c_fro.append(np.linalg.norm(dC) / np.linalg.norm(C))
        c_eig.append((np.abs(np.einsum("bi,bc,ci->i", V, dC, V)) / ev).max())
        np.testing.assert_allclose(mu[j], m, rtol=1e-6)
    return got, max(c_fro), max(c_eig)


@pytest.mark.parametrize("flags", [ALBEDO | SPARSE, ALBEDO | SPARSE | LITERAL])
def test_fp32_at_condition_1e7(scene, flags):
    got, c_fro, c_eig = run_form(scene, flags, FP32)
    assert c_fro < C_FRO_FP32, c_fro
    assert c_eig < C_EIG_FP32, c_eig
    check_alpha(got, scene["ref"], scene["valid"], scene["amp"], TOL_FP32, near=scene["near"])


def test_bf16split_stated_bound_at_condition_1e7(scene):
    got, c_fro, c_eig = run_form(scene, ALBEDO | SPARSE, BF16SPLIT)
    rep = alpha_report(got, scene["ref"], scene["valid"], scene["amp"], near=scene["near"])
    assert c_fro < C_FRO_BF16, c_fro
    assert c_eig < C_EIG_BF16, c_eig
    assert rep["e_2"] < ALPHA_E2_BF16, rep
    assert np.all(got[scene["valid"]] >= 0)
