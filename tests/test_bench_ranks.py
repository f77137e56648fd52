"""The benchmark's multi-process path on CPU: world size 2 over gloo.  Each
rank joins its own points (replicas; no exchange step), the job's time is
the slowest rank's, and the reference arm runs on rank 0 only."""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        got = bench.max_over_ranks(1.5 + 2.0 * rank, dist, "cpu")
        polys, pts, _ = bench.workload("c1", 1000, rank)
        np.save(os.path.join(out, f"pts{rank}.npy"), pts)
        with open(os.path.join(out, f"r{rank}.json"), "w") as f:
            json.dump({"max": got, "n_polys": len(polys), "poly0": np.asarray(polys[0]).tolist()}, f)
    finally:
        dist.destroy_process_group()


def test_two_ranks_gloo(tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    r = [json.load(open(tmp_path / f"r{k}.json")) for k in range(2)]
    assert r[0]["max"] == r[1]["max"] == 3.5              # the slowest rank's time, on every rank
    assert r[0]["n_polys"] == r[1]["n_polys"] and r[0]["poly0"] == r[1]["poly0"]   # same index on every rank
    p0, p1 = np.load(tmp_path / "pts0.npy"), np.load(tmp_path / "pts1.npy")
    assert p0.shape == p1.shape and not np.array_equal(p0, p1)                   # each rank its own points


def test_max_over_ranks_single_process():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(2.25, None, "cpu") == 2.25


def test_reference_arm_other_ranks_exit_quietly():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--gpus", "2", "--n-points", "100000",
                        "--steps", "1", "--warmup", "1"], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip() == ""
