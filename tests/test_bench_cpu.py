"""The measurement script's reference arm runs on the host alone (no GPU): `bench.py --impl
reference` times the oracle and prints one JSON line with the fields the measurement contract
asks for, on the workload the options name."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(*args):
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT,
                         capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    return json.loads(out.stdout.strip().splitlines()[-1])


def test_reference_arm_line():
    d = _run("--impl", "reference", "--steps", "1", "--warmup", "1", "--n", "8")
    assert d["impl"] == "reference"
    assert d["metric"].startswith("rand_cholQR effective HBM GB/s")
    assert d["unit"] == "GB/s" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["steps"] == 1 and d["warmup"] == 1 and d["n_gpus"] == 1
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"] and cb["value"] == d["value"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0
    assert "m=8388608 n=8 " in d["config"]["workload"] and "s1=144 s2=32" in d["config"]["workload"]


def test_reference_arm_takes_the_sketch_sizes():
    d = _run("--impl", "reference", "--steps", "1", "--warmup", "1", "--n", "8", "--s1", "300", "--s2", "40")
    assert "s1=300 s2=40" in d["config"]["workload"]
