"""The multi-rank path of bench.py on CPU with gloo, world size 2: disjoint problem seeds per
rank, the max-over-ranks time and the weak-scaling rate, and the reference arm launched under
torchrun with two ranks printing exactly one line; also the batch size each workload defaults to."""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    elapsed = 1.0 + rank          # rank 1 is the slowest
    m = bench.max_over_ranks(elapsed, "cpu")
    seeds = bench.problem_seeds(4, 100, rank)
    gathered = [None] * world
    dist.all_gather_object(gathered, seeds)
    out[rank] = (m, gathered)
    dist.destroy_process_group()


def test_gloo_world2_max_time_and_disjoint_seeds():
    port = _free_port()
    manager = mp.Manager()
    out = manager.dict()
    mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
    for rank in range(2):
        m, gathered = out[rank]
        assert m == 2.0
        assert len(set(gathered[0]) | set(gathered[1])) == 8
    import bench
    assert bench.weak_scaling_rate(64, 2, 10, 2.0) == 640.0


def test_reference_arm_under_torchrun_two_ranks():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr=127.0.0.1", f"--master-port={port}", "bench.py", "--impl", "reference",
           "--gpus", "2", "--steps", "1", "--warmup", "0"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0


@pytest.mark.parametrize("workload,problems", [("decay512", 152), ("batched", 256), ("order4-krp", 38),
                                               ("order4-kron", 38), ("exact_recovery", 152)])
def test_bench_problem_count_defaults_per_workload(monkeypatch, workload, problems):
    """Without --problems each workload takes the batch its configuration names (order 4: 38 sums,
    which fit one GPU with the autotuner's scratch; batched: 256); --problems overrides it."""
    import bench
    monkeypatch.setattr(sys, "argv", ["bench.py", "--workload", workload])
    assert bench.parse_args().problems == problems
    monkeypatch.setattr(sys, "argv", ["bench.py", "--workload", workload, "--problems", "7"])
    assert bench.parse_args().problems == 7
