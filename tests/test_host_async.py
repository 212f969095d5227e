"""mf_retrieve_host_async: the double-buffered host entry point gives, call
for call, the results of the synchronous host entry point, while calls are
in flight together on one stream."""
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


@pytest.mark.parametrize("precision", [0, 1])
def test_async_host_calls_match_sync(mfg, precision):
    scenes = [workload_scene("plain-512x16x72", seed=s, device="cpu", mask_frac=0.05)
              for s in (1, 2, 3)]
    rows, cols, bands = scenes[0][0].cube.shape
    plan = mfg.Plan(rows, cols, bands, precision=precision)
    ref = []
    for sc, prm in scenes:
        cube = sc.cube.contiguous()
        mask = sc.mask.to(torch.uint8).contiguous()
        ref.append(plan.retrieve_host(cube, sc.k, prm["lam"], prm["eps"], 4, mask=mask).clone())
    # five calls in flight over three scenes (each scene's buffers pinned),
    # alternating the two staging slots, synchronised once at the end
    pinned = [(sc.cube.contiguous().pin_memory(), sc.mask.to(torch.uint8).contiguous().pin_memory(),
               sc.k, prm) for sc, prm in scenes]
    order = [0, 1, 2, 1, 0]
    outs = [torch.empty((rows, cols), dtype=torch.float32).pin_memory() for _ in order]
    stream = torch.cuda.current_stream()
    for i, j in enumerate(order):
        cube, mask, k, prm = pinned[j]
        plan.retrieve_host_async(cube, k, prm["lam"], prm["eps"], 4, mask=mask, out=outs[i],
                                 stream=stream)
    stream.synchronize()
    for i, j in enumerate(order):
        assert torch.equal(outs[i], ref[j]), (i, j)
    plan.close()


def test_async_host_without_mask_and_changing_iterations(mfg):
    scenes = [workload_scene("plain-512x16x72", seed=s, device="cpu") for s in (4, 5)]
    rows, cols, bands = scenes[0][0].cube.shape
    plan = mfg.Plan(rows, cols, bands)
    calls = [(0, 2), (1, 3), (0, 3), (1, 0)]  # (scene, n_iter)
    ref = [plan.retrieve_host(scenes[j][0].cube.contiguous(), scenes[j][0].k,
                              scenes[j][1]["lam"], scenes[j][1]["eps"], n).clone()
           for j, n in calls]
    pinned = [sc.cube.contiguous().pin_memory() for sc, _ in scenes]
    outs = [torch.empty((rows, cols), dtype=torch.float32).pin_memory() for _ in calls]
    for i, (j, n) in enumerate(calls):
        sc, prm = scenes[j]
        plan.retrieve_host_async(pinned[j], sc.k, prm["lam"], prm["eps"], n, out=outs[i])
    torch.cuda.current_stream().synchronize()
    for i in range(len(calls)):
        assert torch.equal(outs[i], ref[i]), i
    plan.close()
