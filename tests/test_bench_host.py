"""The benchmark's reference arm on the CPU: `bench.py --impl reference` times
the FP64 oracle on crops of the workload and prints one JSON line with the
same metric, unit and direction as the GPU arm, plus its CPU-baseline record."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(*args):
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], capture_output=True, text=True,
                       timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout[-2000:]
    return json.loads(lines[0])


def test_reference_arm_line():
    d = _run("--impl", "reference", "--steps", "1", "--warmup", "1")
    sys.path.insert(0, ROOT)
    import bench
    assert d["impl"] == "reference"
    assert d["metric"] == bench.METRIC and d["unit"] == "MPix/s" and d["higher_is_better"] is True
    assert d["value"] > 0 and d["steps"] == 1 and d["n_gpus"] == 1
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["h2d_bytes_per_step"] == 0
    assert d["e2e"]["d2h_bytes_per_step"] == 0
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["config"]["workload"] == bench.WORKLOADS["gray1024"]["desc"]


def test_workload_table():
    sys.path.insert(0, ROOT)
    import bench
    for name, w in bench.WORKLOADS.items():
        assert {"H", "W", "C", "desc", "cpu_crop", "ref_crop"} <= set(w), name
    assert bench.WORKLOADS["pnp64_small"].get("pnp_hi") == 256 and bench.WORKLOADS["pnp64_small"]["pnp"]
