"""The multi-rank host path of bench.py on CPU ranks (gloo backend).

The retrieval does not shard across GPUs beyond independent replicas (one
process per GPU, each on its own flightline, no data-path collective); what
N > 1 adds is host logic: process-group set-up from the launcher's
environment, the barriers around the timed region, the maximum of the
per-rank times, and the reference arm that only rank 0 runs and prints.
"""
import json
import os
import socket
import subprocess
import sys

import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    # CPU ranks: no device may be visible, so that the gloo backend is chosen
    os.environ.update(CUDA_VISIBLE_DEVICES="", RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    w, r, local = bench.dist_init()
    assert (w, r, local) == (world, rank, rank)
    assert dist.get_backend() == "gloo"
    bench.barrier(w)
    # per-rank "step times": every rank must see the slowest one
    m = bench.max_over_ranks(1.5 + 2.0 * rank, w)
    bench.barrier(w)
    with open(f"{out}.{rank}", "w") as f:
        json.dump(m, f)
    dist.destroy_process_group()


def test_max_over_ranks_two_gloo_ranks(tmp_path):
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path / "max")), nprocs=2,
                       start_method="spawn")
    for r in range(2):
        with open(tmp_path / f"max.{r}") as f:
            assert json.load(f) == 3.5


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    env = {k: os.environ.pop(k) for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK") if k in os.environ}
    try:
        assert bench.dist_init() == (1, 0, 0)
        assert bench.max_over_ranks(2.25, 1) == 2.25
        bench.barrier(1)
    finally:
        os.environ.update(env)


def test_reference_arm_under_torchrun_prints_one_line_from_rank_0():
    port = _free_port()
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="", OMP_NUM_THREADS="2")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py",
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0"]
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
    assert line["e2e"]["value"] == line["value"]
    assert line["cpu_baseline"]["kind"] == "oracle"
