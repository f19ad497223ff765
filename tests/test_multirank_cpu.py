"""The benchmark's N > 1 path on the CPU: two gloo ranks, each an
independent replica (the column does not shard), combined into whole-job
figures by the slowest rank's time and the sum of the ranks' work; the
reference arm runs on rank 0 only."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r: (10 + r) ms for 100 (r + 1) bond-steps
        ms, steps = bench.aggregate_over_ranks(10.0 + rank, 100.0 * (rank + 1), dist, "cpu")
        dist.barrier()
        with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
            json.dump({"ms": ms, "bond_steps": steps}, f)
    finally:
        dist.destroy_process_group()


def test_two_replicas_aggregate_by_the_slowest_rank_and_the_total_work(tmp_path):
    import torch.multiprocessing as mp
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       join=True, start_method="spawn")
    for r in range(world):
        got = json.load(open(tmp_path / f"rank{r}.json"))
        # every rank sees the same whole-job figures
        assert got == {"ms": 11.0, "bond_steps": 300.0}


def test_one_process_needs_no_collective():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate_over_ranks(7.5, 42.0, None) == (7.5, 42.0)


def test_reference_arm_runs_on_rank_0_only():
    env = dict(os.environ, RANK="1", LOCAL_RANK="1", WORLD_SIZE="2")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--gpus", "2", "--steps", "1", "--warmup", "3"],
                       capture_output=True, text=True, env=env, timeout=300)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""
