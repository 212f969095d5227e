"""Objective of every iterate (the energy of Fig. 5, Sec. III-B) through the
C ABI (mf_retrieve_energy) against the FP64 oracle's ``retrieve_energy``.

Bar: the energies are sums over a partition's N pixels of O(B) terms, so
E ~ N B.  The CUDA path forms the quadratic part in closed form from its
double-float Woodbury pieces and the per-pixel part in float32 (relative
rounding ~1e-7 per pixel); the moments behind C^k are float32 sums (the
float32 form's C^k is within ~1e-6 relative of the oracle's), which moves E
by about the same relative amount.  1e-5 relative per iterate leaves a margin
of ten over those and is still well below the iterates' decrease."""
import numpy as np
import pytest
import torch

import oracle
from synth import make_scene, workload_scene

pytestmark = pytest.mark.gpu

BF16SPLIT = 1
REL = 1e-5


def _energy(cube_np, k, lam, eps, n_iter, mask=None, col_group=1, flags=3, precision=0):
    import paper_2003_02978_gb300 as mfg
    rows, cols, bt = cube_np.shape
    cube = torch.from_numpy(np.ascontiguousarray(cube_np, np.float32)).cuda()
    m = None if mask is None else torch.from_numpy(np.ascontiguousarray(mask, np.uint8)).cuda()
    plan = mfg.Plan(rows, cols, bt, col_group=col_group, flags=flags, precision=precision)
    a, e = plan.retrieve_energy(cube, np.asarray(k, np.float32), lam, eps, n_iter, mask=m)
    torch.cuda.synchronize()
    st = plan.status()
    plan.close()
    return a.cpu().numpy(), e.cpu().numpy(), st


@pytest.mark.parametrize("precision", [0, BF16SPLIT])
@pytest.mark.parametrize("n_iter", [0, 1, 10])
def test_energy_matches_oracle(precision, n_iter):
    sc, prm = workload_scene("plain-512x16x72", seed=7)
    cube = sc.cube.numpy()
    kk = np.asarray(sc.k, np.float32).astype(np.float64)
    ref = oracle.retrieve_energy(cube.astype(np.float64), kk, prm["lam"], prm["eps"], n_iter)
    _, got, st = _energy(cube, sc.k, prm["lam"], prm["eps"], n_iter, precision=precision)
    assert np.all(st == 0)
    assert got.shape == ref.shape == (16, n_iter + 1)
    np.testing.assert_allclose(got, ref, rtol=REL, atol=0)


def test_energy_grouped_masked():
    """Detector groups with a remainder (Sec. II-E) and masked pixels."""
    sc = make_scene(900, 11, 72, n_plumes=3, plume_sigma=(3.0, 6.0), plume_peak=(1000.0, 4000.0),
                    mask_frac=0.05, seed=5)
    cube, mask = sc.cube.numpy(), sc.mask.numpy()
    kk = np.asarray(sc.k, np.float32).astype(np.float64)
    ref = oracle.retrieve_energy(cube.astype(np.float64), kk, 1e-3, 1e-9, 6, mask=mask,
                                 col_group=4)
    _, got, st = _energy(cube, sc.k, 1e-3, 1e-9, 6, mask=mask, col_group=4)
    assert np.all(st == 0) and got.shape == (3, 7)
    np.testing.assert_allclose(got, ref, rtol=REL, atol=0)


def test_energy_one_partition_converges():
    """All detectors of a flightline grouped into one partition, as in the
    convergence experiment of Fig. 5: the energy settles (its last steps
    change far less than its first ones) and every iterate matches the
    oracle."""
    sc = make_scene(1200, 24, 72, n_plumes=4, plume_sigma=(3.0, 8.0), plume_peak=(1000.0, 5000.0),
                    mask_frac=0.02, seed=9)
    cube, mask = sc.cube.numpy(), sc.mask.numpy()
    kk = np.asarray(sc.k, np.float32).astype(np.float64)
    n = 20
    ref = oracle.retrieve_energy(cube.astype(np.float64), kk, 1e-3, 1e-9, n, mask=mask,
                                 col_group=24)
    _, got, st = _energy(cube, sc.k, 1e-3, 1e-9, n, mask=mask, col_group=24)
    assert np.all(st == 0) and got.shape == (1, n + 1)
    np.testing.assert_allclose(got, ref, rtol=REL, atol=0)
    d = np.abs(np.diff(ref[0]))
    assert d[-5:].max() < 0.05 * d[1:6].max()


def test_energy_rejects_literal_schedule():
    import paper_2003_02978_gb300 as mfg
    plan = mfg.Plan(64, 4, 16, flags=1 | 2 | 4)
    cube = torch.zeros((64, 4, 16), dtype=torch.float32, device="cuda")
    with pytest.raises(mfg.MFError):
        plan.retrieve_energy(cube, np.full(16, -1e-4, np.float32), 1e-3, 1e-9, 2)
