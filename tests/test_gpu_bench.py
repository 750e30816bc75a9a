"""bench.py's JSON line on a small workload: every key of the contract present
and consistent, for the library arm and the reference (oracle) arm."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run_bench(*args):
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT,
                         capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, out.stdout[-2000:]
    return json.loads(lines[0])


def test_bench_line_has_the_contract_keys():
    d = run_bench("--workload", "er10k", "--steps", "3", "--warmup", "3", "--cpu-budget-s", "1",
                  "--stream-count", "40", "--check-workers", "2", "--arena-gib", "1",
                  "--host-staging-gib", "1")
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "e2e",
              "gpu_launches", "roofline", "cpu_baseline", "clocks"):
        assert k in d, k
    assert d["n_gpus"] == 1 and d["steps"] == 3 and d["warmup"] == 3
    assert d["value"] > 0 and d["higher_is_better"] is True and d["scaling"] == "weak"
    assert d["config"]["workload"] and d["gpu_launches"] > 0
    assert d["e2e"]["value"] > 0 and d["e2e"]["h2d_bytes_per_step"] > 0
    r = d["roofline"]
    assert r["bound"] == "hbm" and r["peak"] > 0 and abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-9
    c = d["cpu_baseline"]
    assert c["kind"] == "oracle" and c["cores"] == 1 and c["value"] > 0
    assert "sm_mhz" in d["clocks"] and "reasons" in d["clocks"]
    s = d["stream"]
    assert s["graphs"] == 40 and s["results_checked"] == 40 * len(s["runs"])
    for run in ("one_launch_saturated", "batched_saturated"):
        assert s["runs"][run]["graphs_per_s"] > 0
    for tag in ("at_0.7x_one_launch", "at_0.7x_batched"):
        for server in ("one_launch", "batched"):
            r = s["runs"][f"{server}_{tag}"]
            assert r["p99_ms"] >= r["p50_ms"] > 0


def test_reference_arm_line():
    d = run_bench("--impl", "reference", "--workload", "er10k", "--steps", "3", "--warmup", "3")
    assert d["impl"] == "reference" and d["value"] > 0
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
