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


def test_integer_roofline_arithmetic():
    """The per-pipe bound of the bench's roofline on a hand-computed case:
    one batch of 1,000 pairs, each 100 wavefront cells, 116 character
    compares (one further 16-base window) and 5 backtrace steps, timed at
    1 ms at 2,000 MHz.  Per pair: ALU 100*22 + 1*9 + 5*8 = 2,249, XU 100 + 1
    = 101, shared memory 100*12 + 1*4 + 5*3 = 1,219 (issue: their sum,
    3,569); per-pipe peak = 152 SMs x rate x 2e9 clocks/s.  The binding pipe
    is the one with the longest time: shared memory (1,219 / 32 > 2,249 /
    64 > 101 / 16)."""
    import bench

    class C:
        cells, char_compares, bt_steps = 100_000, 116_000, 5_000

    r = bench.integer_roofline([(1000, C())], [1000], [1.0], 2000.0)
    clk = 152 * 2000e6
    p = r["pipes"]
    assert p["alu"]["ops_per_pair"] == 2249 and p["xu"]["ops_per_pair"] == 101
    assert p["lsu"]["ops_per_pair"] == 1219 and p["issue"]["ops_per_pair"] == 3569
    assert r["pipe"] == "lsu"
    t_lsu = 1219 * 1000 / (32 * clk) * 1e3  # ms at the peak
    assert abs(r["time_ms"] - t_lsu) < 1e-12 and abs(r["frac"] - t_lsu / 1.0) < 1e-12
    assert abs(r["peak"] - 32 * clk / 1e12) < 1e-9
    assert abs(r["achieved"] - 1219 * 1000 / 1e-3 / 1e12) < 1e-9
    # the flat model: 100*32 + 1*18 + 5*12 = 3,278 ops a pair at the issue rate
    assert r["flat"]["ops_per_pair"] == 3278
    assert abs(r["flat"]["frac"] - 3278 * 1000 / (128 * clk) * 1e3 / 1.0) < 1e-12  # ms over the measured 1 ms


def test_traffic_record_matches_the_sources():
    """The DRAM traffic the bench reports comes from an ncu capture of the
    device sources as they stand: the record's digest is the sources', the
    launch-list and counter summaries name the same digest, and the bytes
    per pair lie between the algorithmic input and output (about 248 B) and
    twice that."""
    import bench

    sha = bench.kernel_sources_digest()
    assert bench.NCU_TRAFFIC["sha"] == sha
    for e in (2, 4):
        assert 248 <= bench.NCU_TRAFFIC["bytes_per_pair"][e] <= 2 * 248
    prof = os.path.join(ROOT, "profiles")
    for name in ("launch_list_5Mx100bp_E2_E4.md", "lane_kernel_and_ordering_1Mx100bp_E2_E4_ncu.md"):
        assert sha in open(os.path.join(prof, name)).read(), name
