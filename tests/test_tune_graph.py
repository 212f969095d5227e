"""Launch-shape tuning and CUDA-graph replay: neither changes what is
computed (only the grid decomposition, or how the launches are issued)."""
import json

import numpy as np
import pytest
import torch

import oracle
from parity import check_alpha, f32, retrieve_near_threshold
from synth import workload_scene

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2003_02978_gb300 import build
    build.build()


def test_graph_replay_is_bitwise_equal_to_direct_launches():
    import paper_2003_02978_gb300 as mfg
    sc, prm = workload_scene("plain-512x16x72", seed=2, device="cuda")
    outs = []
    for tuning in ({"use_graph": -1}, {}):
        plan = mfg.Plan(512, 16, 72, tuning=tuning)
        for _ in range(2):  # the second call replays the captured graph
            a = plan.retrieve(sc.cube, sc.k, prm["lam"], prm["eps"], prm["n_iter"])
        torch.cuda.synchronize()
        outs.append(a.cpu().numpy())
        plan.close()
    np.testing.assert_array_equal(outs[0], outs[1])


def test_graph_recaptures_on_new_arguments():
    import paper_2003_02978_gb300 as mfg
    sc, prm = workload_scene("plain-512x16x72", seed=4, device="cuda")
    plan = mfg.Plan(512, 16, 72)
    a3 = plan.retrieve(sc.cube, sc.k, prm["lam"], prm["eps"], 3).clone()
    a5 = plan.retrieve(sc.cube, sc.k, prm["lam"], prm["eps"], 5).clone()
    b3 = plan.retrieve(sc.cube, sc.k, prm["lam"], prm["eps"], 3).clone()
    lam2 = plan.retrieve(sc.cube, sc.k, 10 * prm["lam"], prm["eps"], 3).clone()
    torch.cuda.synchronize()
    assert torch.equal(a3, b3)
    assert not torch.equal(a3, a5)
    assert not torch.equal(a3, lam2)
    cube = sc.cube.cpu().numpy().astype(np.float64)
    for got, lam, n in ((a5, prm["lam"], 5), (lam2, 10 * prm["lam"], 3)):
        ref, _ = oracle.retrieve(cube, f32(sc.k), lam, prm["eps"], n)
        valid = oracle.valid_pixels(sc.cube.cpu().numpy(), None)
        amp = oracle.retrieve_amplification(cube, f32(sc.k), lam, prm["eps"], n)
        near = retrieve_near_threshold(cube, f32(sc.k), lam, prm["eps"], n)
        check_alpha(got.cpu().numpy(), ref, valid, amp, near=near)


def test_autotune_picks_a_candidate_and_caches(tmp_path, monkeypatch):
    import paper_2003_02978_gb300 as mfg
    from paper_2003_02978_gb300 import tune
    monkeypatch.setenv("MF_TUNE_CACHE", str(tmp_path / "tune.json"))
    sc, prm = workload_scene("plain-512x16x72", seed=6, device="cuda")
    best = tune.autotune(sc.cube, sc.k, prm["lam"], prm["eps"], prm["n_iter"], reps=1)
    assert set(best) == {"pixel_rows", "stat_rows", "persistent"}
    assert best["pixel_rows"] in tune.PIXEL_ROWS and best["stat_rows"] in tune.STAT_ROWS
    assert best["persistent"] in (0, 1)
    cache = json.loads((tmp_path / "tune.json").read_text())
    (entry,) = cache.values()
    assert entry["tuning"] == best
    # the shape grid in the launch-per-pass schedule, the default shape in the
    # persistent one
    assert len(entry["candidates"]) == len(tune.PIXEL_ROWS) * len(tune.STAT_ROWS) + 1
    assert sum(c["tuning"]["persistent"] for c in entry["candidates"]) == 1
    # cached: returned without timing again
    assert tune.autotune(sc.cube, sc.k, prm["lam"], prm["eps"], prm["n_iter"]) == best
    # the tuned plan computes the same retrieval (within the float32 bar)
    plan = mfg.Plan(512, 16, 72, tuning=best)
    a = plan.retrieve(sc.cube, sc.k, prm["lam"], prm["eps"], prm["n_iter"])
    torch.cuda.synchronize()
    cube = sc.cube.cpu().numpy().astype(np.float64)
    ref, _ = oracle.retrieve(cube, f32(sc.k), prm["lam"], prm["eps"], prm["n_iter"])
    valid = oracle.valid_pixels(sc.cube.cpu().numpy(), None)
    amp = oracle.retrieve_amplification(cube, f32(sc.k), prm["lam"], prm["eps"], prm["n_iter"])
    near = retrieve_near_threshold(cube, f32(sc.k), prm["lam"], prm["eps"], prm["n_iter"])
    check_alpha(a.cpu().numpy(), ref, valid, amp, near=near)
    plan.close()
