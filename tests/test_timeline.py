"""The device timeline (mf_timeline): per-launch spans of a retrieval as it
runs, graph replay included, read without changing what the retrieval
computes."""
import numpy as np
import pytest
import torch

from synth import workload_scene

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mfg():
    from paper_2003_02978_gb300 import build
    build.build()
    import paper_2003_02978_gb300 as m
    return m


@pytest.mark.parametrize("precision,literal", [(1, False), (0, False), (0, True)])
def test_timeline_spans_every_launch(mfg, precision, literal):
    sc, prm = workload_scene("flightline-4000x598x72", seed=0, device="cuda")
    rows, cols, bands = sc.cube.shape
    n_iter = 4
    k = torch.as_tensor(np.asarray(sc.k, np.float32), device="cuda")
    flags = mfg.ALBEDO | mfg.SPARSE | (mfg.LITERAL if literal else 0)
    plan = mfg.Plan(rows, cols, bands, flags=flags, precision=precision)
    ref = plan.retrieve(sc.cube, k, prm["lam"], prm["eps"], n_iter, mask=sc.mask).clone()
    plan.timeline(True)
    got = []
    for _ in range(2):  # the capture, then a replay of the captured graph
        a = plan.retrieve(sc.cube, k, prm["lam"], prm["eps"], n_iter, mask=sc.mask)
        spans = plan.timeline_read()
        got.append(a.clone())
        kinds = [s[0] for s in spans]
        # pilot + statistics, initial solve, then per pass (solve, pixel); the
        # literal schedule adds a statistics pass and its solve per iteration
        if literal:
            expect = ["stats", "stats", "solve", "pixel"] + \
                ["solve", "stats", "solve", "pixel"] * n_iter
        else:
            expect = ["stats", "stats", "solve", "pixel"] + ["solve", "pixel"] * n_iter
        assert kinds == expect
        # one stream: every launch starts after the previous one ended
        prev_end = None
        for kind, t0, t1 in spans:
            assert t0 is not None and t1 is not None and t1 > t0
            if prev_end is not None:
                assert t0 >= prev_end
            prev_end = t1
        assert spans[0][1] == 0.0
        pixel = [t1 - t0 for kind, t0, t1 in spans if kind == "pixel"]
        assert all(5.0 < d < 5e4 for d in pixel), pixel
    plan.timeline(False)
    a = plan.retrieve(sc.cube, k, prm["lam"], prm["eps"], n_iter, mask=sc.mask)
    assert plan.timeline_read() == []
    # the probes change no result
    for g in got + [a]:
        assert torch.equal(g, ref)
    plan.close()
