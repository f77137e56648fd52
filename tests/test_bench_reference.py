"""The benchmark's reference arm (the CPU oracle, timed on the host) runs
without a GPU and prints one JSON line whose metric, unit and workload are the
GPU arm's."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--n-points", "100000", "--steps", "1",
                        "--warmup", "1"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference"
    assert line["unit"] == "points/s" and line["higher_is_better"] is True and line["value"] > 0
    assert line["config"]["workload"] == "c2-city-300polys-mixture-points-1e05"
    assert line["config"]["n_points_per_gpu"] == 100000 and line["config"]["polygons"] == 300
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": "points/s", "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
