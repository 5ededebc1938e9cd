"""The reference arm of bench.py on the CPU: the FP64 oracle timed on the host cores
prints one JSON line with the benchmark's metric, unit and workload, the oracle as
its cpu_baseline and an e2e entry with no host-device bytes; a second rank prints
nothing and exits 0."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run_bench(*extra, env=None):
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                           "--warmup", "0", *extra], cwd=ROOT, capture_output=True, text=True, timeout=600,
                          env=env)


def test_reference_arm_json_line():
    sys.path.insert(0, ROOT)
    import bench
    r = run_bench()
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    out = json.loads(lines[0])
    assert out["impl"] == "reference"
    assert out["metric"] == bench.METRIC and out["unit"] == "Msamples/s"
    assert out["config"]["workload"] == bench.WORKLOAD
    assert out["higher_is_better"] is True and out["value"] > 0
    cb = out["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == out["value"] and cb["sample"]
    assert out["e2e"] == {"value": out["value"], "unit": "Msamples/s", "h2d_bytes_per_step": 0,
                          "d2h_bytes_per_step": 0}


def test_reference_arm_other_rank_is_silent():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = run_bench("--gpus", "2", env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip() == ""
