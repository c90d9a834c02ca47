"""The benchmark's JSON contract, checked on the CPU: the reference arm (the
oracle on the host cores) prints one line with the same metric, unit and
config as the GPU arm; under a multi-rank launch only rank 0 prints."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _run(extra_env, *argv):
    env = dict(os.environ, **extra_env)
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *argv], cwd=ROOT, env=env,
                          capture_output=True, text=True, timeout=600)


def test_headline_config_counts_both_batches():
    c = bench.headline_config(5_000_000, 1)
    assert c["pairs_per_step_per_gpu"] == 10_000_000
    assert c["parallelism"] == "replicas x1"
    assert "E=2% and E=4%" in c["workload"] and "both batches" in c["workload"]
    one = bench.headline_config(1_000, 4, (4,))
    assert one["pairs_per_step_per_gpu"] == 1_000 and one["parallelism"] == "replicas x4"
    assert "E=4%" in one["workload"] and "E=2%" not in one["workload"]


def test_reference_arm_line():
    r = _run({}, "--impl", "reference", "--steps", "1", "--warmup", "3", "--pairs", "2000")
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"] == bench.METRIC and d["unit"] == "pairs/s" and d["higher_is_better"] is True
    assert d["config"] == bench.headline_config(2000, 1)
    assert d["steps"] == 1 and d["warmup"] == 3 and d["value"] > 0
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "pairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


@pytest.mark.parametrize("rank", [1, 3])
def test_reference_arm_other_ranks_print_nothing(rank):
    r = _run({"RANK": str(rank), "WORLD_SIZE": "4", "LOCAL_RANK": str(rank)}, "--impl", "reference", "--steps", "1",
             "--warmup", "3", "--pairs", "2000")
    assert r.returncode == 0, r.stderr[-2000:]
    assert not [ln for ln in r.stdout.splitlines() if ln.startswith("{")]


def test_clock_records_that_void_a_number():
    ok = {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 4}
    assert not bench.clocks_rejected(ok)
    assert not bench.clocks_rejected(dict(ok, reasons=["sw_power_cap"], sm_mhz=1900.0))
    for r in ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"):
        assert bench.clocks_rejected(dict(ok, reasons=[r]))
    assert bench.clocks_rejected(dict(ok, sm_mhz=1200.0))  # stuck low, no reason: a leftover lock
    assert not bench.clocks_rejected(dict(ok, sm_mhz=1200.0, reasons=["sw_power_cap"]))
    assert not bench.clocks_rejected({"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]})
    assert not bench.clocks_rejected(None)
