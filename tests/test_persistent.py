"""Persistent form (MF_PERSISTENT): after the statistics pass one launch runs
the initial solves, every pixel pass and every iteration solve of every line
as work items of a dependency-ordered queue.  Each item runs the same device
code as the launch-per-pass sequence, so the two agree bit for bit; the
persistent form is also compared with the FP64 oracle line by line, and its
bounded waits are made to run out (on the host's request, no GPU fault)."""
import numpy as np
import pytest
import torch

from parity import TOL_FP32, f32
from synth import batched_lines, make_scene, workload_scene
from test_batched import check_lines, make_batch

pytestmark = pytest.mark.gpu

ALBEDO, SPARSE, PERSISTENT = 1, 2, 16


def same_bits(a, b):
    """Equal bit patterns (the NaN of a failed partition included)."""
    return a.shape == b.shape and torch.equal(a.contiguous().view(torch.int32),
                                              b.contiguous().view(torch.int32))


@pytest.fixture(scope="module")
def mfg():
    from paper_2003_02978_gb300 import build
    build.build()
    import paper_2003_02978_gb300 as m
    return m


def _pair(mfg, line_rows, cols, bands, cube, mask, k, lams, n_iters, precision=0, col_group=1,
          flags=ALBEDO | SPARSE, repeat=1):
    """alpha and status of the sequence and of the persistent form (the last
    of `repeat` calls, so that graph replay is covered)."""
    out = []
    for extra in (0, PERSISTENT):
        plan = mfg.BatchPlan(line_rows, cols, bands, col_group=col_group, flags=flags | extra,
                             precision=precision)
        for _ in range(repeat):
            a = plan.retrieve(cube.cuda(), k, lams, 1e-9, n_iters, mask=mask.cuda())
        torch.cuda.synchronize()
        out.append((a.cpu().clone(), plan.status()))
        plan.close()
    return out


@pytest.mark.parametrize("precision", [0, 1])
def test_queue_equals_sequence_uneven_lines(mfg, precision):
    # lines of uneven length, one with no iterations, per-line lambda
    line_rows = [1100, 1300, 1000, 1700, 1500]
    lams = [1e-3, 1e-4, 3e-3, 1e-3, 1e-2]
    n_iters = [3, 5, 0, 2, 4]
    _, cube, mask, k = make_batch(line_rows, 40, 72, seed=11)
    (a_seq, st_seq), (a_q, st_q) = _pair(mfg, line_rows, 40, 72, cube, mask, k, lams, n_iters,
                                         precision=precision, repeat=2)
    np.testing.assert_array_equal(st_q, st_seq)
    assert same_bits(a_q, a_seq)


def test_queue_col_groups_across_tiles(mfg):
    # 5-column partitions: partition 3 (columns 15-19) spans two 16-column
    # tiles, so its solves wait on two tiles and both tiles on it
    line_rows = [900, 1400, 700]
    _, cube, mask, k = make_batch(line_rows, 40, 72, seed=23)
    (a_seq, st_seq), (a_q, st_q) = _pair(mfg, line_rows, 40, 72, cube, mask, k,
                                         [1e-3, 2e-3, 5e-4], [2, 4, 3], col_group=5)
    np.testing.assert_array_equal(st_q, st_seq)
    assert same_bits(a_q, a_seq)


def test_queue_single_line_and_changing_iterations(mfg):
    sc, prm = workload_scene("plain-512x16x72", seed=2, mask_frac=0.05)
    cube, mask = sc.cube.cuda(), sc.mask.cuda()
    seq = mfg.Plan(512, 16, 72)
    que = mfg.Plan(512, 16, 72, flags=ALBEDO | SPARSE | PERSISTENT)
    for n_iter in (4, 0, 1, 6):
        a = seq.retrieve(cube, sc.k, prm["lam"], prm["eps"], n_iter, mask=mask).clone()
        b = que.retrieve(cube, sc.k, prm["lam"], prm["eps"], n_iter, mask=mask).clone()
        torch.cuda.synchronize()
        assert same_bits(a, b), n_iter
        assert np.all(que.status() == 0)
    seq.close()
    que.close()


def test_queue_failed_line_and_energy(mfg):
    """A line too short for its covariance fails alone (NOT_SPD, NaN), as in
    the sequence; the per-iterate energy agrees bit for bit."""
    line_rows = [500, 40, 600]
    _, cube, mask, k = make_batch(line_rows, 6, 72, seed=3, mask_frac=0.0)
    (a_seq, st_seq), (a_q, st_q) = _pair(mfg, line_rows, 6, 72, cube, mask, k, [1e-3] * 3,
                                         [3, 3, 3])
    assert np.all(st_q[6:12] == 4) and np.all(st_q[:6] == 0) and np.all(st_q[12:] == 0)
    np.testing.assert_array_equal(st_q, st_seq)
    assert same_bits(a_q, a_seq)
    sc, prm = workload_scene("plain-512x16x72", seed=4, mask_frac=0.05)
    res = []
    for extra in (0, PERSISTENT):
        plan = mfg.Plan(512, 16, 72, flags=ALBEDO | SPARSE | extra)
        a, en = plan.retrieve_energy(sc.cube.cuda(), sc.k, prm["lam"], prm["eps"], 5,
                                     mask=sc.mask.cuda())
        torch.cuda.synchronize()
        res.append((a.cpu(), en.cpu()))
        plan.close()
    assert same_bits(res[0][0], res[1][0])
    assert torch.equal(res[0][1].view(torch.int64), res[1][1].view(torch.int64))


@pytest.mark.parametrize("precision", [0, 1])
def test_queue_oracle_parity(mfg, precision):
    """Lines drawn like the batched workload (per-column masked fraction
    U(0, 0.3), lambda log-uniform in [1e-4, 1e-2], N_iter in 5..20), every
    partition against the FP64 oracle."""
    lines = batched_lines(4, cols=12, rows_range=(1500, 3000), seed=8)
    scenes = [make_scene(ln["rows"], 12, 72, n_plumes=3, plume_sigma=(3.0, 8.0),
                         plume_peak=(500.0, 5000.0), mask_col_frac=ln["mask_col_frac"],
                         seed=ln["seed"]) for ln in lines]
    cube = torch.cat([s.cube for s in scenes], 0).contiguous()
    mask = torch.cat([s.mask for s in scenes], 0).contiguous()
    k = f32(scenes[0].k)
    rows = [ln["rows"] for ln in lines]
    lams = [ln["lam"] for ln in lines]
    nits = [ln["n_iter"] for ln in lines]
    plan = mfg.BatchPlan(rows, 12, 72, flags=ALBEDO | SPARSE | PERSISTENT, precision=precision)
    a = plan.retrieve(cube.cuda(), k, lams, 1e-9, nits, mask=mask.cuda())
    torch.cuda.synchronize()
    got, status, slices = a.cpu().numpy(), plan.status(), plan.line_slices()
    plan.close()
    assert np.all(status == 0)
    # the BF16-split form's stated per-pixel bound for partitions of 1000 to
    # 2000 valid pixels (as in the launch-per-pass batched tests)
    check_lines(scenes, cube, mask, k, got, status, slices, lams, nits, ALBEDO | SPARSE, TOL_FP32,
                tol_pix=2e-4 if precision else None)


@pytest.mark.parametrize("precision", [0, 1])
def test_queue_timeline_is_one_launch(mfg, precision):
    sc, prm = workload_scene("plain-512x16x72", seed=5)
    plan = mfg.Plan(512, 16, 72, flags=ALBEDO | SPARSE | PERSISTENT, precision=precision)
    plan.timeline(True)
    for _ in range(2):  # capture, then replay
        plan.retrieve(sc.cube.cuda(), sc.k, prm["lam"], prm["eps"], 3)
        spans = plan.timeline_read()
        # pilot, statistics, then the work queue
        assert [s[0] for s in spans] == ["stats", "stats", "queue"]
        assert spans[2][1] >= spans[1][2]
    plan.close()


def test_queue_wait_runs_out_and_context_survives(mfg, monkeypatch):
    """MF_FAULT=timeout: every pixel item of the first pass makes a bounded
    wait on a barrier nothing arrives on, takes the timeout path (its copies
    land first) and raises the abort word; the items waiting on those pixel
    items see it and leave.  Every partition reports MF_ERR_TIMEOUT, and
    plans made afterwards retrieve as before."""
    sc, prm = workload_scene("plain-512x16x72", seed=6, mask_frac=0.05)
    cube, mask = sc.cube.cuda(), sc.mask.cuda()
    monkeypatch.setenv("MF_FAULT", "timeout")
    bad = mfg.Plan(512, 16, 72, flags=ALBEDO | SPARSE | PERSISTENT)
    monkeypatch.delenv("MF_FAULT")
    bad.retrieve(cube, sc.k, prm["lam"], prm["eps"], 3, mask=mask)
    torch.cuda.synchronize()
    assert np.all(bad.status() == 6)
    bad.close()
    seq = mfg.Plan(512, 16, 72)
    que = mfg.Plan(512, 16, 72, flags=ALBEDO | SPARSE | PERSISTENT)
    a = seq.retrieve(cube, sc.k, prm["lam"], prm["eps"], 3, mask=mask).clone()
    b = que.retrieve(cube, sc.k, prm["lam"], prm["eps"], 3, mask=mask).clone()
    torch.cuda.synchronize()
    assert same_bits(a, b) and np.all(que.status() == 0)
    seq.close()
    que.close()


def test_queue_rejects_literal(mfg):
    with pytest.raises(mfg.MFError):
        mfg.Plan(512, 16, 72, flags=ALBEDO | SPARSE | PERSISTENT | 4)


def test_queue_checkpointed_forward_and_gradients(mfg):
    """The differentiation form's forward (checkpoints of every pass) through
    the work queue: alpha and the gradients the adjoint computes from the
    checkpoint agree bit for bit with the launch-per-pass forward."""
    sc, prm = workload_scene("plain-512x16x72", seed=7, mask_frac=0.05)
    cube, mask = sc.cube.cuda(), sc.mask.cuda()
    rng = np.random.default_rng(0)
    g = torch.as_tensor(rng.standard_normal((512, 16)), dtype=torch.float32).cuda()
    res = []
    for extra in (0, PERSISTENT):
        plan = mfg.Plan(512, 16, 72, flags=ALBEDO | SPARSE | extra)
        alpha, ck = plan.retrieve_train(cube, np.asarray(f32(sc.k), np.float32), prm["lam"],
                                        prm["eps"], 4, mask=mask, cube_grad=True)
        gk, gl, gc = plan.backward(ck, g, cube_grad=True)
        torch.cuda.synchronize()
        res.append([t.detach().cpu().clone() for t in (alpha, gk, gl.reshape(1), gc)])
        assert np.all(plan.status() == 0)
        plan.close()
    for a, b in zip(res[0], res[1]):
        assert same_bits(a, b)
