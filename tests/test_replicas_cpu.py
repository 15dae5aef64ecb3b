"""The multi-GPU path of the benchmark is "replicas only" (one independent lattice per rank, no data-path
collective): the job time is the largest rank time and the value the sum of the ranks' node updates.
Checked here on CPU with two gloo ranks; the reference arm under torchrun runs on rank 0 alone."""
import json
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, results):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_ms = 10.0 + 5.0 * rank  # rank 1 is the slow replica
    ms = bench.max_over_ranks(local_ms, dist, "cpu")
    value = bench.replica_value(world, 1000, 2, 50, ms * 1e-3)
    results[rank] = (ms, value)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_replicas_take_the_slowest_time():
    import torch.multiprocessing as mp
    port = _free_port()
    with mp.Manager() as man:
        results = man.dict()
        mp.spawn(_rank, args=(2, port, results), nprocs=2, join=True)
        res = dict(results)
    assert res[0] == res[1]
    ms, value = res[0]
    assert ms == 15.0
    # two lattices of 1000 nodes x 2 species x 50 steps in 15 ms
    assert value == pytest.approx(2 * 1000 * 2 * 50 / 0.015 / 1e6)


def test_reference_arm_under_torchrun_runs_on_rank_zero_only():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0"]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle"
