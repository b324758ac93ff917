"""The measurement script's reference arm runs on the host alone (no GPU): `bench.py --impl
reference` times the oracle and prints one JSON line with the fields the measurement contract
asks for, on the workload the options name."""
import json
import os
import subprocess
import sys

import pytest

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


def test_roofline_fields_from_a_launch_time():
    # the dominant kernel's roofline object: algorithmic bytes per launch over the launch time,
    # against the measured copy peak, with the DRAM traffic scaled from the capture
    import bench
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if not os.path.exists(path):
        pytest.skip("no measured peaks on this machine")
    peak = json.load(open(path))["hbm_gbs"]
    m, n = 1 << 23, 64
    r = bench.kernel_roofline("trsm_tc", 2.5, m, n)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and r["peak"] == peak
    assert abs(r["achieved"] - 16 * n * m / 2.5e-3 / 1e9) < 1e-6
    assert abs(r["frac"] - r["achieved"] / peak) < 1e-12
    assert r["traffic"] == bench.MEASURED_DRAM_BYTES_PER_ROW_N64["trsm_tc"] * m
    assert bench.kernel_roofline("trsm_tc", 2.5, m, 32)["traffic"] is None  # captured at n = 64 only


def test_workload_names_carry_the_sketch_sizes():
    import argparse
    import bench
    a = argparse.Namespace(m=1 << 23, n=64, kappa=1e12, s1=0, s2=0)
    assert bench.sketch_sizes(a) == (8320, 256)
    assert bench.workload_name(a) == "rand_cholQR m=8388608 n=64 kappa=1e+12 s1=8320 s2=256"
    a.s1, a.s2 = 34279, 776
    assert bench.workload_name(a).endswith("s1=34279 s2=776")


def test_dominant_roofline_is_taken_per_solve():
    # n = 128: a solve is four block launches, so the solve's roofline divides its bytes by the
    # time of a whole solve, not of one launch (per launch it would read above the copy peak)
    import bench
    if not os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")):
        pytest.skip("no measured peaks on this machine")
    m, n, steps = 1 << 23, 128, 5
    kt = {"trsm_tc": (20.0 * steps, 8 * steps), "gram_tc": (6.5 * steps, 2 * steps),
          "cs_scatter": (2.0 * steps, steps)}
    r = bench.dominant_roofline(kt, 30.0, steps, m, n)
    assert r["kernel"] == "trsm_tc"
    assert abs(r["achieved"] - 16 * n * m / 10.0e-3 / 1e9) < 1e-6  # two solves of 10 ms each
    assert abs(r["kernel_share"] - 20.0 / 30.0) < 1e-12
    # a kind without a unit is taken per launch
    r = bench.dominant_roofline({"hhqr": (3.0 * steps, steps)}, 30.0, steps, m, n)
    assert r["kernel"] == "hhqr" and r["achieved"] is None
