"""Batched form: many flightlines of uneven length, stacked along rows, in one
retrieval (every kernel covers all lines), each line with its own partitions,
lambda and iteration count.  Each line's alpha is compared with the FP64
oracle run on that line alone."""
import numpy as np
import pytest
import torch

import oracle
from parity import TOL_FP32, check_alpha, f32, retrieve_near_threshold
from synth import make_scene

pytestmark = pytest.mark.gpu

ALBEDO, SPARSE, LITERAL = 1, 2, 4


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2003_02978_gb300 import build
    build.build()


def make_batch(line_rows, cols, bands, seed, mask_frac=0.03, nan_masked=False):
    scenes = [make_scene(r, cols, bands, n_plumes=2, plume_sigma=(3.0, 6.0),
                         plume_peak=(800.0, 3000.0), mask_frac=mask_frac, nan_masked=nan_masked,
                         seed=seed + 17 * i) for i, r in enumerate(line_rows)]
    cube = torch.cat([s.cube for s in scenes], 0).contiguous()
    mask = torch.cat([s.mask if s.mask is not None else
                      torch.zeros(s.cube.shape[:2], dtype=torch.uint8) for s in scenes],
                     0).contiguous()
    k = f32(scenes[0].k)  # one target spectrum for the whole batch
    return scenes, cube, mask, k


def run_batch(line_rows, cols, bands, cube, mask, k, lams, n_iters, flags=ALBEDO | SPARSE,
              precision=0, col_group=1):
    import paper_2003_02978_gb300 as mfg
    plan = mfg.BatchPlan(line_rows, cols, bands, col_group=col_group, flags=flags,
                         precision=precision)
    a = plan.retrieve(cube.cuda(), k, lams, 1e-9, n_iters, mask=mask.cuda())
    torch.cuda.synchronize()
    out = a.cpu().numpy(), plan.status(), plan.line_slices(), plan.P
    plan.close()
    return out


def check_lines(scenes, cube, mask, k, got, status, slices, lams, n_iters, flags, tol,
                col_group=1, tol_pix=None):
    cube = cube.numpy()
    mask = mask.numpy()
    pl = -(-cube.shape[1] // col_group)
    for li, sl in enumerate(slices):
        sub, msk = cube[sl], mask[sl]
        ref, st = oracle.retrieve(sub.astype(np.float64), k, lams[li], 1e-9, n_iters[li],
                                  mask=msk, flags=flags, col_group=col_group)
        np.testing.assert_array_equal(status[li * pl:(li + 1) * pl], st)
        valid = oracle.valid_pixels(sub, msk)
        ok = valid.copy()
        for pi in np.nonzero(st)[0]:
            ok[:, pi * col_group:(pi + 1) * col_group] = False
        assert np.all(got[sl][~valid] == 0)
        amp = oracle.retrieve_amplification(sub.astype(np.float64), k, lams[li], 1e-9,
                                            n_iters[li], mask=msk, flags=flags,
                                            col_group=col_group)
        near = retrieve_near_threshold(sub.astype(np.float64), k, lams[li], 1e-9, n_iters[li],
                                       mask=msk, flags=flags, col_group=col_group)
        check_alpha(got[sl], ref, ok, amp, tol, near=near, tol_pix=tol_pix)


# (a line of 260 rows, 3.6 samples per band, leaves C so ill-conditioned that
# float32 pixel dot products miss the bar at lambda = 1e-2, as a single-line
# plan does (measured e_2 3.4e-4); the float32 lines keep N >= 4 B, the
# BF16-split ones N >= 10 B.  A single BF16-split iteration from a 1700-row
# line has pixels amplified 244-fold by the reweighting map, whose errors
# dominate e_2 (1.2e-4, single-line plan alike): that line runs 2 iterations.
# The BF16-split bound of 1e-4 is stated for partitions of at least 1000 valid
# pixels (the batched workload's lines have 2000 to 30000 rows): a 760-row
# line measured e_inf 1.8e-4, e_2 5.1e-5, single-line plan alike)
BATCH_CASES = {
    0: ([300, 700, 517, 1100, 560], [1e-3, 1e-4, 3e-3, 1e-3, 1e-2], [3, 5, 0, 1, 4]),
    1: ([1100, 1300, 1000, 1700, 1500], [1e-3, 1e-4, 3e-3, 1e-3, 1e-2], [3, 5, 0, 2, 4]),
}


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_uneven_lines(precision):
    line_rows, lams, n_iters = BATCH_CASES[precision]
    scenes, cube, mask, k = make_batch(line_rows, 9, 72, seed=41)
    got, status, slices, P = run_batch(line_rows, 9, 72, cube, mask, k, lams, n_iters,
                                       precision=precision)
    assert P == 5 * 9
    check_lines(scenes, cube, mask, k, got, status, slices, lams, n_iters, ALBEDO | SPARSE,
                TOL_FP32)


def test_batch_literal_and_groups():
    line_rows = [400, 900, 650]
    lams = [1e-3, 2e-3, 5e-4]
    n_iters = [2, 4, 3]
    scenes, cube, mask, k = make_batch(line_rows, 11, 72, seed=7)
    got, status, slices, P = run_batch(line_rows, 11, 72, cube, mask, k, lams, n_iters,
                                       flags=ALBEDO | SPARSE | LITERAL, col_group=3)
    assert P == 3 * 4
    check_lines(scenes, cube, mask, k, got, status, slices, lams, n_iters,
                ALBEDO | SPARSE | LITERAL, TOL_FP32, col_group=3)


def test_batch_short_line_fails_alone():
    """A line with fewer valid pixels per column than bands fails (NOT_SPD,
    NaN alpha) without touching the other lines."""
    line_rows = [500, 40, 600]
    lams = [1e-3] * 3
    n_iters = [3, 3, 3]
    scenes, cube, mask, k = make_batch(line_rows, 6, 72, seed=3, mask_frac=0.0)
    got, status, slices, P = run_batch(line_rows, 6, 72, cube, mask, k, lams, n_iters)
    assert np.all(status[6:12] == 4) and np.all(status[:6] == 0) and np.all(status[12:] == 0)
    assert np.all(np.isnan(got[slices[1]]))
    check_lines([scenes[0]], cube[:500], mask[:500], k, got[:500], status[:6], [slice(0, 500)],
                lams[:1], n_iters[:1], ALBEDO | SPARSE, TOL_FP32)


def test_batch_matches_single_line_plans():
    """Each line of a batch equals the same line retrieved on its own plan
    within the float32 bar (the chunking of the statistics may differ)."""
    import paper_2003_02978_gb300 as mfg
    line_rows = [640, 1280]
    scenes, cube, mask, k = make_batch(line_rows, 16, 72, seed=5)
    got, status, slices, _ = run_batch(line_rows, 16, 72, cube, mask, k, [1e-3, 2e-3], [4, 6])
    for li, sl in enumerate(slices):
        plan = mfg.Plan(line_rows[li], 16, 72)
        a = plan.retrieve(cube[sl].contiguous().cuda(), k, [1e-3, 2e-3][li], 1e-9, [4, 6][li],
                          mask=mask[sl].contiguous().cuda())
        torch.cuda.synchronize()
        single = a.cpu().numpy()
        valid = oracle.valid_pixels(cube[sl].numpy(), mask[sl].numpy())
        d = np.abs(got[sl] - single)[valid]
        assert d.max() <= 1e-4 * np.abs(single[valid]).max()
        plan.close()


def test_batch_rejects_bad_rows():
    import paper_2003_02978_gb300 as mfg
    with pytest.raises(mfg.MFError):
        mfg.BatchPlan([100, 0, 50], 4, 72)


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_per_column_mask_fraction(precision):
    """Lines drawn like the batched workload (synth.batched_lines): per-column
    masked fraction U(0, 0.3), lambda log-uniform in [1e-4, 1e-2], N_iter in
    5..20; shorter lines and fewer columns so that the oracle checks every
    partition.  Lines keep at least 1500 rows, so that every partition has
    the 1000 valid pixels the BF16-split bound is stated for."""
    from synth import batched_lines, make_scene
    lines = batched_lines(4, cols=12, rows_range=(1500, 3000), seed=3)
    # the BF16-split form's stated per-pixel bound for partitions of 1000 to
    # 2000 valid pixels: 2e-4 of max|alpha| (e_2 stays within 1e-4)
    tol_pix = 2e-4 if precision else None
    scenes = [make_scene(ln["rows"], 12, 72, n_plumes=3, plume_sigma=(3.0, 8.0),
                         plume_peak=(500.0, 5000.0), mask_col_frac=ln["mask_col_frac"],
                         seed=ln["seed"]) for ln in lines]
    cube = torch.cat([s.cube for s in scenes], 0).contiguous()
    mask = torch.cat([s.mask for s in scenes], 0).contiguous()
    k = f32(scenes[0].k)
    rows = [ln["rows"] for ln in lines]
    lams = [ln["lam"] for ln in lines]
    nits = [ln["n_iter"] for ln in lines]
    got, status, slices, P = run_batch(rows, 12, 72, cube, mask, k, lams, nits,
                                       precision=precision)
    assert P == 4 * 12 and np.all(status == 0)
    check_lines(scenes, cube, mask, k, got, status, slices, lams, nits, ALBEDO | SPARSE, TOL_FP32,
                tol_pix=tol_pix)
