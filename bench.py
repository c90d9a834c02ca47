"""Benchmark: batched exact gap-affine WFA of the paper's workload on GB300.

Workload (paper Sec. II: 5 million pairs of 100 bp reads at edit-distance
thresholds E = 2 % and 4 %): per GPU, two synthetic batches of 5,000,000
pairs of 100 bp (2 and 4 edits), penalties x=4, o=6, e=2, score + CIGAR.
A step aligns both batches (10 M pairs per GPU).

value : pairs/s with inputs already resident in HBM (device-pointer call),
        timed with CUDA events on the launching stream.
e2e   : the same through the host-pointer call (pinned host buffers; the
        library's host->device and device->host copies inside the timed
        region).
roofline : the short-read wavefront kernel (the dominant kernel), its
        algorithmic work per launch over its event-timed duration.
cpu_baseline : the plain CPU oracle on the host cores, bounded sample.

Run: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Multi-GPU: launched by torchrun; each rank aligns its own shard (weak
scaling, replicas, no data collective).
"""

from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "pairs/s 100bp E=2%/4% (score+CIGAR) batched vs plain, % roofline; p99 latency"
PEN = (4, 6, 2)
N_PAIRS = 5_000_000
LENGTH = 100
EDITS = (2, 4)
SEED = 1
CIGAR_WORDS_PER_PAIR = 16
PEAKS_FALLBACK = {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}
N_SM = 152
# Integer work of the method, per unit and instruction class: a wavefront
# cell is the three recurrences (three
# maxima, two +1, three sequence-end tests with their selects) and one
# 16-base extension window (two word indices, two funnel shifts, XOR,
# count-leading-zeros, halving, the advance and its end clamp); its shared
# memory traffic is the five source offsets, the three results and the four
# packed words of the window.  A further window repeats the window part; a
# backtrace step reads the three candidates of its cell and picks one.
WORK = {"cell": {"alu": 22, "xu": 1, "lsu": 12},
        "window": {"alu": 9, "xu": 1, "lsu": 4},
        "bt_step": {"alu": 8, "xu": 0, "lsu": 3}}
# per-SM throughput of each class in lanes per clock on sm_100-class SMs:
# the integer ALU pipe (add, min/max, compare, select, logic, shifts) 64, the
# XU pipe (count leading zeros) 16, shared-memory accesses 32 (one warp-wide
# access a clock), instruction issue 128 (four schedulers x 32 lanes)
PIPE_RATE = {"alu": 64, "xu": 16, "lsu": 32, "issue": 128}
# the flat model of earlier measurements: every op at the issue rate
FLAT_OPS = {"cell": 32, "window": 18, "bt_step": 12}
# DRAM traffic of the short-read path (dram__bytes_read.sum +
# dram__bytes_write.sum from ncu on 1M-pair launches of the same workload, per
# pair, the ordering pass and the lane kernel added; the traffic of a launch
# grows in proportion to its pairs), valid for the device sources whose
# digest is "sha" (kernel_sources_digest); any change to them voids it
NCU_TRAFFIC = {"sha": "f07ac210ffcba225", "bytes_per_pair": {2: 276.94 + 137.18, 4: 278.07 + 148.94}}
# the kernels of the timed region at the time of that capture
NCU_KERNEL = "lane_order_kernel + lane_kernel"
KERNEL_SOURCES = ("wfa_device.cuh", "short_path.cuh", "arena_path.cuh", "lane_path.cuh", "kernels.cu", "launch.h")


def kernel_sources_digest() -> str:
    import hashlib

    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "paper_2204_02085_gb300", "csrc", f),
                  "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--pairs", type=int, default=N_PAIRS, help="pairs per batch (default: the paper's 5M)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample", type=int, default=N_PAIRS, help="pairs per edit rate for the CPU baseline")
    ap.add_argument("--edits", default="2,4", help="edit counts of the batches (default: the paper's 2%% and 4%%)")
    ap.add_argument("--short-variant", type=int, default=None,
                    help="force one short-read kernel variant (tuning; default: the library's autotuner)")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-pointer (end-to-end) measurement")
    ap.add_argument("--no-numa-bind", action="store_true",
                    help="do not restrict the process to the GPU's local CPUs before allocating page-locked buffers")
    ap.add_argument("--no-samples", action="store_true",
                    help="skip the bounded mixed-length and serving samples of the default run")
    ap.add_argument("--mixed-pairs", type=int, default=200_000, help="pairs of the mixed-length sample")
    ap.add_argument("--serving-requests", type=int, default=400, help="requests of the serving sample")
    ap.add_argument("--arena-gb", type=float, default=None,
                    help="scratch arena size for configs 3 and 4 (default: 16 and 64 GiB)")
    ap.add_argument("--requests", type=int, default=2000, help="requests in the serving trace (config 5)")
    ap.add_argument("--workers", type=int, default=2, help="server slots (config 5)")
    ap.add_argument("--baselines", type=int, default=1, help="config 5: also replay the one-at-a-time baselines")
    ap.add_argument("--config", type=int, default=2, choices=[2, 3, 4, 5, 6],
                    help="2: the paper's 5M x 100 bp workload (default); 3: 1M mixed-length pairs (100-2,000 bp, "
                         "0-10%% edits, tandem repeats); 4: 20k long-read pairs (10 kbp, 1-5%% edits); 5: serving, "
                         "a Poisson stream of requests")
    args = ap.parse_args()
    args.edits = tuple(int(e) for e in args.edits.split(","))
    return args


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            p = json.load(f)
        return p, "measured"
    return dict(PEAKS_FALLBACK), "fallback"


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while running."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for name, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# throttle reasons that void a timed region's number
REJECT_REASONS = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown")


def clocks_rejected(clk) -> bool:
    """True when a timed region's clock record voids its number: a hardware
    or thermal slowdown was active, or the SM clock sat well below its
    maximum with no reason given (a clock lock left behind).  sw_power_cap
    alone is kept (and reported)."""
    if not clk or clk.get("sm_mhz") is None:
        return False
    reasons = clk.get("reasons") or []
    if any(r in REJECT_REASONS for r in reasons):
        return True
    smax = clk.get("sm_max_mhz")
    return bool(smax) and clk["sm_mhz"] < 0.85 * smax and not reasons


def make_batches(n_pairs: int, rank: int, edits=EDITS):
    from paper_2204_02085_gb300 import sharding, synth

    return [synth.uniform_reads(n_pairs, LENGTH, e, seed=sharding.shard_seed(SEED, rank)) for e in edits]


def cpu_oracle_run(batches, sample: int, threads: int | None = None):
    """The oracle (plain CPU WFA, score + CIGAR) on the first `sample` pairs
    of each batch, all host cores (or `threads`).  Returns (pairs, seconds,
    threads, [(pairs, counters) per batch])."""
    import oracle
    from paper_2204_02085_gb300 import synth

    oracle.build()
    threads = threads or host_cores()
    pairs = 0
    cnts = []
    t0 = time.perf_counter()
    for b in batches:
        k = min(sample, b.n)
        sub = synth.Batch(b.patterns, b.pattern_offsets[:k], b.pattern_lengths[:k], b.texts, b.text_offsets[:k],
                          b.text_lengths[:k])
        cnt = oracle.Counts()
        oracle.wfa_batch(sub, PEN, nthreads=threads, runs_per_pair=64, counts=cnt)
        cnts.append((k, cnt))
        pairs += k
    dt = time.perf_counter() - t0
    return pairs, dt, threads, cnts


def integer_roofline(cnts, n_launch, ms_launch, sm_mhz: float) -> dict:
    """The integer-issue bound of the short kernel's launches from the
    oracle's counters ([(pairs counted, Counts)] per batch), the pairs and
    measured milliseconds of each launch, and the SM clock.  Per pair: cells,
    further 16-base windows ((compares - cells) / 16) and backtrace steps,
    times WORK per class; each class at its pipe's rate (PIPE_RATE), the
    slowest pipe binding.  Also the flat model (every op at the issue rate)."""
    clk = N_SM * sm_mhz * 1e6  # SM clocks per second, summed over SMs
    pipes = {p: {"ops_per_pair": 0.0, "time_ms": 0.0} for p in PIPE_RATE}
    flat_ops, flat_ms, meas_ms = 0.0, 0.0, 0.0
    for (k, c), n, ms in zip(cnts, n_launch, ms_launch):
        units = {"cell": c.cells / k, "window": max(0.0, (c.char_compares - c.cells) / 16.0) / k,
                 "bt_step": c.bt_steps / k}
        per = {p: sum(units[u] * WORK[u].get(p, 0) for u in units) for p in ("alu", "xu", "lsu")}
        per["issue"] = sum(per.values())
        for p, v in per.items():
            pipes[p]["ops_per_pair"] += v * n
            pipes[p]["time_ms"] += v * n / (PIPE_RATE[p] * clk) * 1e3
        fo = sum(units[u] * FLAT_OPS[u] for u in units)
        flat_ops += fo * n
        flat_ms += fo * n / (PIPE_RATE["issue"] * clk) * 1e3
        meas_ms += ms
    ntot = float(sum(n_launch))
    for p, d in pipes.items():
        d["peak"] = PIPE_RATE[p] * clk / 1e12
        d["achieved"] = d["ops_per_pair"] / (meas_ms / 1e3) / 1e12
        d["frac"] = d["time_ms"] / meas_ms
        d["ops_per_pair"] /= ntot
    bind = max(pipes, key=lambda p: pipes[p]["time_ms"])
    b = pipes[bind]
    flat = {"ops_per_pair": flat_ops / ntot, "peak": PIPE_RATE["issue"] * clk / 1e12,
            "achieved": flat_ops / (meas_ms / 1e3) / 1e12, "frac": flat_ms / meas_ms, "unit": "Tops/s"}
    return {"bound": "alu", "pipe": bind, "achieved": b["achieved"], "peak": b["peak"], "unit": "Tops/s",
            "frac": b["frac"], "time_ms": b["time_ms"], "measured_ms": meas_ms, "pipes": pipes, "flat": flat,
            "peak_source": "152 SMs x lanes per clock of the pipe (ALU 64, XU 16, shared memory 32, issue 128) x "
                           "%.0f MHz" % sm_mhz,
            "work_per_unit": WORK}


def headline_config(n_pairs: int, world: int, edits=EDITS) -> dict:
    """The headline workload's config (both arms print the same one)."""
    rates = " and ".join("E=%d%%" % e for e in edits)
    return {"workload": "%d pairs x %d bp per batch, %s (%s edits), penalties 4/6/2, score+CIGAR; one step = "
                        "%s" % (n_pairs, LENGTH, rates, " and ".join(str(e) for e in edits),
                                "both batches" if len(edits) == 2 else "%d batch(es)" % len(edits)),
            "pairs_per_step_per_gpu": len(edits) * n_pairs, "parallelism": "replicas x%d" % world,
            "l2": "inputs larger than L2 (about %.1f GB of ASCII per batch)" % (2 * n_pairs * LENGTH / 1e9)}


def run_reference(args):
    """--impl reference: the oracle, as it stands, timed on the host cores
    (rank 0 only); each step is a bounded sample of the same workload."""
    from paper_2204_02085_gb300 import sharding

    rank, world, _ = sharding.dist_env()
    if rank != 0:
        return 0
    sample = min(100_000, args.pairs)
    batches = make_batches(sample, 0, args.edits)
    for _ in range(args.warmup):
        cpu_oracle_run(batches, sample)
    t_total, pairs_total, threads = 0.0, 0, host_cores()
    for _ in range(args.steps):
        p, dt, threads, _ = cpu_oracle_run(batches, sample)
        t_total += dt
        pairs_total += p
    value = pairs_total / t_total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "pairs/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * t_total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic",
        "config": headline_config(args.pairs, world, args.edits),
        "cpu_baseline": {"value": value, "unit": "pairs/s", "cores": threads, "kind": "oracle",
                         "sample": "each step the first %d pairs of each batch (E=2%%, E=4%%)" % sample},
        "e2e": {"value": value, "unit": "pairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_config(args):
    """Configurations beside the headline one (rank 0 only): mixed-length
    pairs (3) and long reads (4), timed like the headline workload with
    device-resident inputs; long reads both score-only and score + CIGAR."""
    import torch

    import paper_2204_02085_gb300 as pkg
    from paper_2204_02085_gb300 import build as gpu_build
    from paper_2204_02085_gb300 import synth

    gpu_build.build()
    dev = torch.device("cuda:0")
    if args.config == 3:
        n = args.pairs if args.pairs != N_PAIRS else 1_000_000
        b = synth.mixed_reads(n, 100, 2000, 0.10, 0.05, seed=3)
        scratch, modes = 16 << 30, (False,)
        workload = "%d pairs, text length log-uniform 100-2,000 bp, edit rate U[0,10%%], 5%% tandem repeats" % n
    else:
        n = args.pairs if args.pairs != N_PAIRS else 20_000
        b = synth.long_reads(n, 10_000, 0.01, 0.05, seed=4)
        scratch, modes = 64 << 30, (True, False)
        workload = "%d pairs x 10 kbp, edit rate U[1%%,5%%]" % n
    if args.arena_gb is not None:
        scratch = int(args.arena_gb * (1 << 30))
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    d = dict(pat=t(b.patterns), plen=t(b.pattern_lengths), txt=t(b.texts), tlen=t(b.text_lengths),
             s=torch.empty(n, dtype=torch.int32, device=dev), st=torch.empty(n, dtype=torch.int8, device=dev),
             off=torch.empty(n + 1, dtype=torch.int64, device=dev))
    stream = torch.cuda.Stream(dev)
    res = {}
    runs = [(so, {}) for so in modes]
    if args.config == 3:  # batched (graph replay) and the plain baseline beside the eager path
        runs = [(False, {}), (False, dict(graph=True)), (False, dict(plain=True))]
    with pkg.Aligner(0, scratch_bytes=scratch) as al:
        al.set_stream(stream)
        for score_only, extra in runs:
            w = torch.empty(1, dtype=torch.int32, device=dev)
            if not score_only:  # size the CIGAR output from a first call
                al.align_device(d["pat"], None, d["plen"], d["txt"], None, d["tlen"], d["s"], d["st"], w, d["off"],
                                pen=PEN)
                w = torch.empty(int(d["off"][-1]) + 1, dtype=torch.int32, device=dev)

            def call():
                rc = al.align_device(d["pat"], None, d["plen"], d["txt"], None, d["tlen"], d["s"], d["st"],
                                     None if score_only else w, d["off"], pen=PEN, score_only=score_only,
                                     timing=True, **extra)
                assert rc == pkg.WFA_GPU_OK
                return al.timing()

            for _ in range(args.warmup):
                call()
            torch.cuda.synchronize(dev)
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ts = []
            ev0.record(stream)
            for _ in range(args.steps):
                ts.append(call())
            ev1.record(stream)
            torch.cuda.synchronize(dev)
            ms = ev0.elapsed_time(ev1) / args.steps
            st = d["st"].cpu().numpy()
            label = "score_only" if score_only else "score_cigar"
            if extra:
                label += "_" + "_".join(k for k in extra)
            res[label] = {
                "pairs_per_s": n / (ms / 1000.0), "ms_per_call": ms,
                "phase_ms": {k: round(float(np.mean([x[k] for x in ts])), 3)
                             for k in ("align_ms", "general_ms", "cigar_ms", "total_ms")},
                "deferred_pairs": int(ts[-1]["deferred_pairs"]), "short_variant": int(ts[-1]["short_variant"]),
                "status_ok": int((st == 0).sum()), "mean_score": float(d["s"].float().mean().item())}
    main_mode = res.get("score_cigar_graph") or res.get("score_cigar")
    if "score_cigar_plain" in res:
        res["batched_over_plain"] = main_mode["pairs_per_s"] / res["score_cigar_plain"]["pairs_per_s"]
    line = {"metric": "pairs/s (config %d)" % args.config, "value": main_mode["pairs_per_s"], "unit": "pairs/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": main_mode["ms_per_call"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic", "config": {"workload": workload, "penalties": "4/6/2",
                                            "arena_bytes": scratch}, "modes": res}
    print(json.dumps(line), flush=True)
    return 0


def run_models(args):
    """Configuration 6: the other penalty models and ends-free alignment
    (rank 0 only), device-resident inputs, score + CIGAR: 5M x 100 bp pairs
    at E=4% (seed 1) under gap-affine 4/6/2, edit distance (1/0/1: the
    M-only short kernel) and gap-linear 3/0/2; 1M 100 bp reads (3 edits)
    against reference windows of 100-300 bp (seed 6), global and with the
    text ends free (semi-global)."""
    import torch

    import paper_2204_02085_gb300 as pkg
    from paper_2204_02085_gb300 import build as gpu_build
    from paper_2204_02085_gb300 import synth

    gpu_build.build()
    dev = torch.device("cuda:0")
    n_short = args.pairs if args.pairs != N_PAIRS else N_PAIRS
    n_win = max(1, n_short // 5)
    work = {"reads_100bp_E4": synth.uniform_reads(n_short, LENGTH, 4, seed=SEED),
            "reads_in_windows": synth.reads_in_windows(n_win, 100, 100, 3, seed=6)}
    runs = [("reads_100bp_E4", "gap_affine_4_6_2", (4, 6, 2), (0, 0, 0, 0)),
            ("reads_100bp_E4", "edit_distance_1_0_1", (1, 0, 1), (0, 0, 0, 0)),
            ("reads_100bp_E4", "gap_linear_3_0_2", (3, 0, 2), (0, 0, 0, 0)),
            ("reads_in_windows", "global_4_6_2", (4, 6, 2), (0, 0, 0, 0)),
            ("reads_in_windows", "text_ends_free_4_6_2", (4, 6, 2), (0, 0, 300, 300))]
    stream = torch.cuda.Stream(dev)
    res = {}
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)  # noqa: E731
    with pkg.Aligner(0, scratch_bytes=8 << 30) as al:
        al.set_stream(stream)
        for wname, label, pen, ends in runs:
            b = work[wname]
            n = b.n
            d = dict(pat=t(b.patterns), plen=t(b.pattern_lengths), txt=t(b.texts), tlen=t(b.text_lengths),
                     s=torch.empty(n, dtype=torch.int32, device=dev), st=torch.empty(n, dtype=torch.int8, device=dev),
                     off=torch.empty(n + 1, dtype=torch.int64, device=dev))
            al.set_ends_free(*ends)
            w = torch.empty(1, dtype=torch.int32, device=dev)
            al.align_device(d["pat"], None, d["plen"], d["txt"], None, d["tlen"], d["s"], d["st"], w, d["off"],
                            pen=pen)
            w = torch.empty(int(d["off"][-1]) + 1, dtype=torch.int32, device=dev)

            def call():
                rc = al.align_device(d["pat"], None, d["plen"], d["txt"], None, d["tlen"], d["s"], d["st"], w,
                                     d["off"], pen=pen, timing=True)
                assert rc == pkg.WFA_GPU_OK
                return al.timing()

            for _ in range(args.warmup):
                call()
            torch.cuda.synchronize(dev)
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ts = []
            ev0.record(stream)
            for _ in range(args.steps):
                ts.append(call())
            ev1.record(stream)
            torch.cuda.synchronize(dev)
            ms = ev0.elapsed_time(ev1) / args.steps
            res[label] = {"workload": wname, "pairs": n, "pairs_per_s": n / (ms / 1000.0), "ms_per_call": ms,
                          "ends_free": ends,
                          "short_kernel_ms": round(float(np.mean([x["align_ms"] for x in ts])), 3),
                          "arena_ms": round(float(np.mean([x["general_ms"] for x in ts])), 3),
                          "short_variant": al.variant_name(int(ts[-1]["short_variant"])),
                          "deferred_pairs": int(ts[-1]["deferred_pairs"]),
                          "mean_score": float(d["s"].float().mean().item())}
            del d
    main = res["edit_distance_1_0_1"]
    line = {"metric": "pairs/s (config 6: penalty models, ends-free)", "value": main["pairs_per_s"],
            "unit": "pairs/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": main["ms_per_call"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "int32", "data": "synthetic",
            "config": {"workload": "%d x 100 bp pairs at E=4%% under three penalty models; %d 100 bp reads "
                                   "against 100-300 bp windows, global and text-ends-free" % (n_short, n_win)},
            "modes": res}
    print(json.dumps(line), flush=True)
    return 0


def serving_experiment(R: int, workers: int, burst: bool = True, one: bool = True, plain: bool = True) -> dict:
    """Configuration 5's trace: a Poisson stream of R requests (2,000 per
    second; batch sizes log-uniform 1-4,096 pairs; lengths log-uniform
    100-5,000 bp; edit rate U[2%, 8%]; seed 5) replayed in real time against
    the continuous-batching server (`workers` slots; queued requests of the
    same parameters are merged into one call); then, if asked, all queued at
    once (capacity), and without a server: one request at a time in arrival
    order on the default path and on the plain path (the baseline of issuing
    each batch to the plain kernels).  Requests are windows of a pool of
    page-locked pairs, built before the clock starts."""
    import threading as th

    import torch

    import paper_2204_02085_gb300 as pkg
    from paper_2204_02085_gb300 import synth

    rng = np.random.Generator(np.random.PCG64(5))
    pool_n = 60_000
    pool = synth.mixed_reads(pool_n, 100, 5000, 0.08, 0.0, seed=5, rate_lo=0.02)

    def pin(a):
        t = torch.empty(a.shape, dtype={np.uint8: torch.uint8, np.int32: torch.int32,
                                         np.int64: torch.int64}[a.dtype.type], pin_memory=True)
        t.numpy()[...] = a
        return t.numpy()

    pool = synth.Batch(pin(pool.patterns), pin(pool.pattern_offsets), pin(pool.pattern_lengths), pin(pool.texts),
                       pin(pool.text_offsets), pin(pool.text_lengths))
    gaps = rng.exponential(1.0 / 2000.0, size=R)
    arrivals = np.cumsum(gaps) - gaps[0]
    sizes = np.minimum(np.exp(rng.uniform(0, np.log(4096), size=R)).astype(np.int64), pool_n)
    starts = rng.integers(0, pool_n - sizes + 1)
    reqs = []
    for a0, n in zip(starts, sizes):
        sl = slice(int(a0), int(a0 + n))
        reqs.append(synth.Batch(pool.patterns, pool.pattern_offsets[sl], pool.pattern_lengths[sl], pool.texts,
                                pool.text_offsets[sl], pool.text_lengths[sl]))
    caps = [int(b.pattern_lengths.sum() + b.text_lengths.sum()) + 1 for b in reqs]
    total_pairs = int(sizes.sum())

    def replay(workers, burst=False):
        with pkg.Server(0, workers=workers, memory_budget_bytes=32 << 30) as srv:
            # warm-up, untimed: kernels loaded, then a burst so that every
            # slot grows its buffers to merged-batch size
            for b, c in zip(reqs[:4], caps[:4]):
                srv.wait(srv.submit(b, PEN, cigar_capacity=c))
            for rid in [srv.submit(b, PEN, cigar_capacity=c) for b, c in zip(reqs[:256], caps[:256])]:
                srv.wait(rid)
            ids, stats = [None] * R, [None] * R
            done = th.Event()

            def waiter():
                for j in range(R):
                    while ids[j] is None:
                        time.sleep(0.0001)
                    stats[j] = srv.wait(ids[j])[1]
                done.set()

            w = th.Thread(target=waiter)
            w.start()
            t0 = time.perf_counter()
            for j in range(R):
                delay = arrivals[j] - (time.perf_counter() - t0)
                if delay > 0 and not burst:
                    time.sleep(delay)
                ids[j] = srv.submit(reqs[j], PEN, cigar_capacity=caps[j])
            done.wait()
            w.join()
        lat = np.array([(s.end_s - s.submit_s) * 1000.0 for s in stats])
        span = max(s.end_s for s in stats) - min(s.submit_s for s in stats)
        calls = len({(s.worker, s.start_s) for s in stats})
        return {"workers": workers, "calls": calls, "pairs_per_call": total_pairs / calls,
                "p50_ms": float(np.percentile(lat, 50)),
                "p99_ms": float(np.percentile(lat, 99)), "mean_ms": float(lat.mean()),
                "pairs_per_s": total_pairs / span, "span_s": span,
                "all_ok": all(s.result == pkg.WFA_GPU_OK for s in stats)}

    def one_at_a_time(plain):
        """The same trace served without a server: one request at a time in
        arrival order, each aligned alone (default or plain path)."""
        with pkg.Aligner(0, 16 << 30) as al:
            for b, c in zip(reqs[:4], caps[:4]):
                al.align(b, PEN, cigar_capacity=c, plain=plain)
            lat = np.empty(R)
            t0 = time.perf_counter()
            for j in range(R):
                delay = arrivals[j] - (time.perf_counter() - t0)
                if delay > 0:
                    time.sleep(delay)
                al.align(reqs[j], PEN, cigar_capacity=caps[j], plain=plain)
                lat[j] = (time.perf_counter() - t0 - arrivals[j]) * 1000.0
            span = time.perf_counter() - t0
        return {"workers": 1, "plain": plain, "calls": R, "pairs_per_call": total_pairs / R,
                "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                "mean_ms": float(lat.mean()), "pairs_per_s": total_pairs / span, "span_s": span, "all_ok": True}

    out = {"requests": R, "offered_pairs": total_pairs,
           "offered_pairs_per_s": total_pairs / float(arrivals[-1] or 1.0),
           "serving": replay(workers)}
    if burst:
        out["saturated"] = replay(workers, burst=True)  # every request queued at once: capacity
    if one:
        out["one_at_a_time"] = one_at_a_time(False)
    if plain:
        out["plain_per_batch"] = one_at_a_time(True)
        out["p99_plain_over_serving"] = out["plain_per_batch"]["p99_ms"] / out["serving"]["p99_ms"]
    return out


def run_serving(args):
    """Configuration 5 (serving): see serving_experiment; rank 0 only."""
    from paper_2204_02085_gb300 import build as gpu_build

    gpu_build.build()
    R = args.requests
    res = serving_experiment(R, args.workers, burst=True, one=bool(args.baselines), plain=bool(args.baselines))
    serving = res["serving"]
    line = {"metric": "pairs/s and p50/p99 latency (config 5, serving)", "value": serving["pairs_per_s"],
            "unit": "pairs/s", "n_gpus": 1, "steps": R, "warmup": 260, "ms_per_step": serving["mean_ms"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic",
            "config": {"workload": "%d requests, Poisson 2,000/s, batch sizes log-uniform 1-4,096, lengths "
                                   "log-uniform 100-5,000 bp, edit rate U[2%%,8%%], penalties 4/6/2, score+CIGAR"
                                   % R, "offered_pairs": res["offered_pairs"],
                       "offered_pairs_per_s": res["offered_pairs_per_s"]},
            **{k: v for k, v in res.items() if k not in ("requests", "offered_pairs", "offered_pairs_per_s")}}
    print(json.dumps(line), flush=True)
    return 0


def mixed_sample(n: int, steps: int, warmup: int) -> dict:
    """The first n pairs of configuration 3 (text length log-uniform
    100-2,000 bp, edit rate U[0, 10%], 5% tandem repeats, seed 3), device
    resident, score + CIGAR, through the batched path (graph replay), the
    eager path and the plain baseline: pairs/s of each."""
    import torch

    import paper_2204_02085_gb300 as pkg
    from paper_2204_02085_gb300 import synth

    dev = torch.device("cuda:0")
    b = synth.mixed_reads(n, 100, 2000, 0.10, 0.05, seed=3)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)  # noqa: E731
    d = dict(pat=t(b.patterns), plen=t(b.pattern_lengths), txt=t(b.texts), tlen=t(b.text_lengths),
             s=torch.empty(n, dtype=torch.int32, device=dev), st=torch.empty(n, dtype=torch.int8, device=dev),
             off=torch.empty(n + 1, dtype=torch.int64, device=dev))
    stream = torch.cuda.Stream(dev)
    res = {}
    with pkg.Aligner(0, scratch_bytes=16 << 30) as al:
        al.set_stream(stream)
        w = torch.empty(1, dtype=torch.int32, device=dev)
        al.align_device(d["pat"], None, d["plen"], d["txt"], None, d["tlen"], d["s"], d["st"], w, d["off"], pen=PEN)
        w = torch.empty(int(d["off"][-1]) + 1, dtype=torch.int32, device=dev)
        ref = None
        for mode, extra in (("batched", dict(graph=True)), ("eager", {}), ("plain", dict(plain=True))):
            def call():
                rc = al.align_device(d["pat"], None, d["plen"], d["txt"], None, d["tlen"], d["s"], d["st"], w,
                                     d["off"], pen=PEN, timing=True, **extra)
                assert rc == pkg.WFA_GPU_OK
                return al.timing()
            for _ in range(warmup):
                call()
            torch.cuda.synchronize(dev)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ts = []
            e0.record(stream)
            for _ in range(steps):
                ts.append(call())
            e1.record(stream)
            torch.cuda.synchronize(dev)
            ms = e0.elapsed_time(e1) / steps
            sc = d["s"].cpu().numpy()
            if ref is None:
                ref = sc.copy()
            assert np.array_equal(ref, sc), "modes disagree on the mixed sample"
            res[mode] = {"pairs_per_s": n / (ms / 1000.0), "ms_per_call": ms,
                         "short_kernel_ms": round(float(np.mean([x["align_ms"] for x in ts])), 3),
                         "arena_ms": round(float(np.mean([x["general_ms"] for x in ts])), 3),
                         "deferred_pairs": int(ts[-1]["deferred_pairs"]),
                         "short_variant": al.variant_name(int(ts[-1]["short_variant"]))}
    res["batched_over_plain"] = res["batched"]["pairs_per_s"] / res["plain"]["pairs_per_s"]
    res["workload"] = ("first %d pairs of the mixed-length configuration (100-2,000 bp, 0-10%% edits, 5%% "
                       "tandem repeats, seed 3), score+CIGAR, %d timed calls per mode" % (n, steps))
    return res


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.config == 5:
        return run_serving(args)
    if args.config == 6:
        return run_models(args)
    if args.config != 2:
        return run_config(args)

    import torch
    import torch.distributed as dist

    import paper_2204_02085_gb300 as pkg
    from paper_2204_02085_gb300 import build as gpu_build
    from paper_2204_02085_gb300 import hostnuma, sharding

    rank, world, local = sharding.dist_env()
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", init_method="env://")
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)
    # page-locked buffers land on the node of the allocating thread's CPU:
    # run on the GPU's own node before allocating any
    numa = {"bound": False, "skipped": True} if args.no_numa_bind else hostnuma.bind_to_gpu(dev.index)
    if rank == 0 or not os.path.exists(pkg.LIB_PATH):
        gpu_build.build()
    sharding.barrier()

    batches = make_batches(args.pairs, rank, args.edits)
    if args.short_variant is not None:
        os.environ["WFA_GPU_SHORT_VARIANT"] = str(args.short_variant)
    # one non-default stream for the library's work and the timing events
    stream = torch.cuda.Stream(dev)
    al = pkg.Aligner(dev.index)
    al.set_stream(stream)

    # device-resident inputs and outputs
    def to_dev(a):
        return torch.from_numpy(np.ascontiguousarray(a)).to(dev)

    dbat = []
    for b in batches:
        n = b.n
        dbat.append(dict(
            pat=to_dev(b.patterns), plen=to_dev(b.pattern_lengths), txt=to_dev(b.texts), tlen=to_dev(b.text_lengths),
            s=torch.empty(n, dtype=torch.int32, device=dev), st=torch.empty(n, dtype=torch.int8, device=dev),
            off=torch.empty(n + 1, dtype=torch.int64, device=dev),
            w=torch.empty(CIGAR_WORDS_PER_PAIR * n, dtype=torch.int32, device=dev)))

    torch.cuda.synchronize(dev)

    # modes: "batched" = the default path with each batch's device work
    # replayed from a CUDA graph (captured on the first call); "eager" = the
    # default path launched call by call; "plain" = the baseline (the same
    # kernels call by call with one fixed variant: no sampling autotuner, no
    # longest-first order, no graph); "arena_only" = every pair on one-warp
    # arena teams, no short-read kernel
    MODES = {"batched": dict(graph=True), "eager": {}, "plain": dict(plain=True),
             "arena_only": dict(arena_only=True)}

    def device_step(mode, collect=None):
        for d in dbat:
            rc = al.align_device(d["pat"], None, d["plen"], d["txt"], None, d["tlen"], d["s"], d["st"], d["w"],
                                 d["off"], pen=PEN, timing=True, **MODES[mode])
            if rc != pkg.WFA_GPU_OK:
                raise RuntimeError("CIGAR capacity too small: %d words needed" % int(d["off"][-1]))
            if collect is not None:
                collect.append(al.timing())

    def timed(mode, steps, sample_clocks=False):
        for _ in range(args.warmup):
            device_step(mode)
        torch.cuda.synchronize(dev)
        sampler = ClockSampler(dev.index) if (rank == 0 and sample_clocks) else None
        if sampler:
            sampler.start()
        ts = []
        sharding.barrier()
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            device_step(mode, ts)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        sharding.barrier()
        clk = sampler.stop() if sampler else None
        return sharding.max_over_ranks(e0.elapsed_time(e1)), ts, clk

    ms, timings, clocks = timed("batched", args.steps, sample_clocks=True)
    # a rejected clock record: measured once more (every rank takes part; the
    # decision is rank 0's, which samples the clocks)
    if sharding.max_over_ranks(1.0 if clocks_rejected(clocks) else 0.0) > 0:
        first = clocks
        ms, timings, clocks = timed("batched", args.steps, sample_clocks=True)
        clocks = dict(clocks or {}, remeasured=True, first=first)
    pairs_per_step = sum(b.n for b in batches)
    # aligned bases per step: sum over pairs of (n + m) / 2
    bases_per_step = sum(float(b.pattern_lengths.sum()) + float(b.text_lengths.sum()) for b in batches) / 2.0
    value = pairs_per_step * world * args.steps / (ms / 1000.0)
    other_modes = {}
    for mode, steps in (("eager", args.steps), ("plain", args.steps), ("arena_only", max(2, args.steps // 4))):
        mms, mts, _ = timed(mode, steps)
        other_modes[mode] = {"pairs_per_s": pairs_per_step * world * steps / (mms / 1000.0),
                             "ms_per_step": mms / steps, "steps": steps,
                             "align_kernel_ms": [round(float(np.mean([t["align_ms"] for t in mts[i::len(batches)]])),
                                                       3) for i in range(len(batches))],
                             "arena_ms": [round(float(np.mean([t["general_ms"] for t in mts[i::len(batches)]])), 3)
                                          for i in range(len(batches))]}
    device_step("batched")  # the outputs read below come from the headline mode
    torch.cuda.synchronize(dev)

    # per-edit-rate figures and the dominant kernel
    per_batch = {}
    for i, b in enumerate(batches):
        ts = timings[i::len(batches)]
        align_ms = float(np.mean([t["align_ms"] for t in ts]))
        total_ms = float(np.mean([t["total_ms"] for t in ts]))
        per_batch[args.edits[i]] = dict(align_ms=align_ms, total_ms=total_ms,
                                   deferred=int(np.mean([t["deferred_pairs"] for t in ts])),
                                   launches=int(ts[0]["kernel_launches"]),
                                   variant=int(ts[-1]["short_variant"]))
    launches = int(sum(t["kernel_launches"] for t in timings))

    # outputs of the last step, for the work model and a sanity check
    outs = []
    for d in dbat:
        s = d["s"].cpu().numpy()
        st = d["st"].cpu().numpy()
        off = d["off"].cpu().numpy()
        outs.append((s, st, off))
        assert np.all(st == 0), "unexpected pair status in the benchmark workload"

    # ---- e2e: host-pointer calls (pinned host memory) ------------------
    pinned = []
    for b, (s, st, off) in zip(batches if not args.no_e2e else [], outs):
        def pin(a):
            t = torch.empty(a.shape, dtype=getattr(torch, str(a.dtype)) if a.dtype != np.uint8 else torch.uint8,
                            pin_memory=True)
            t.numpy()[...] = a
            return t.numpy()
        n = b.n
        pinned.append(dict(pat=pin(b.patterns), plen=pin(b.pattern_lengths), txt=pin(b.texts),
                           tlen=pin(b.text_lengths),
                           s=torch.empty(n, dtype=torch.int32, pin_memory=True).numpy(),
                           st=torch.empty(n, dtype=torch.int8, pin_memory=True).numpy(),
                           off=torch.empty(n + 1, dtype=torch.int64, pin_memory=True).numpy(),
                           w=torch.empty(CIGAR_WORDS_PER_PAIR * n, dtype=torch.int32, pin_memory=True).numpy()))

    def host_step():
        h2d = d2h = 0
        for p in pinned:
            n = len(p["plen"])
            rc = pkg.wfa_gpu_align_batch(al.ctx, n, p["pat"].ctypes.data, None, p["plen"].ctypes.data,
                                         p["txt"].ctypes.data, None, p["tlen"].ctypes.data, PEN, 0,
                                         pkg.WFA_GPU_TIMING, p["s"].ctypes.data, p["st"].ctypes.data,
                                         p["w"].ctypes.data, p["w"].size, p["off"].ctypes.data)
            if rc != pkg.WFA_GPU_OK:
                raise pkg.WfaGpuError(rc, "e2e align")
            e2e_phases.append(al.timing())
            h2d += p["pat"].nbytes + p["txt"].nbytes + p["plen"].nbytes + p["tlen"].nbytes
            d2h += p["s"].nbytes + p["st"].nbytes + p["off"].nbytes + 4 * int(p["off"][-1])
        return h2d, d2h

    e2e_phases = []
    e2e_steps = 0 if args.no_e2e else max(3, args.steps // 4)
    for _ in range(max(1, args.warmup) if e2e_steps else 0):
        host_step()
    h2d = d2h = 0
    # clocks during the end-to-end region too: a slow process shows whether
    # the GPU's clock or the link was the cause
    e2e_sampler = ClockSampler(dev.index) if (rank == 0 and e2e_steps) else None
    if e2e_sampler:
        e2e_sampler.start()
    sharding.barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        h2d, d2h = host_step()
    e2e_s = sharding.max_over_ranks(time.perf_counter() - t0)
    e2e_clocks = e2e_sampler.stop() if e2e_sampler else None
    e2e_value = pairs_per_step * world * e2e_steps / e2e_s if e2e_steps else None
    if pinned:
        numa["pinned_pages_per_node"] = {str(k): v for k, v in sorted(hostnuma.placement(
            [a.ctypes.data for p in pinned for a in p.values()]).items())}
    if e2e_steps:
        for p, (s, st, off) in zip(pinned, outs):
            assert np.array_equal(p["s"], s) and np.array_equal(p["off"], off), "host and device calls disagree"

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return 0

    # ---- CPU baseline (oracle) and the work model from its counters -----
    peaks, peak_src = load_peaks()
    cpu = None
    cnt = None
    if not args.no_cpu_baseline:
        cp, cdt, cthreads, cnt = cpu_oracle_run(batches, min(args.cpu_sample, args.pairs))
        one = min(100_000, args.pairs)
        cp1, cdt1, _, _ = cpu_oracle_run(batches, one, threads=1)
        cpu = {"value": cp / cdt, "unit": "pairs/s", "cores": cthreads, "kind": "oracle",
               "sample": "first %d pairs of each of the two 5M-pair batches (E=2%%, E=4%%), score+CIGAR, "
                         "%d threads, %.1f s wall" % (min(args.cpu_sample, args.pairs), cthreads, cdt),
               "single_thread": {"value": cp1 / cdt1, "unit": "pairs/s",
                                 "sample": "first %d pairs of each batch, 1 thread, %.1f s" % (one, cdt1)}}

    # algorithmic bytes per pair: 2L ASCII in, lengths in, score + status +
    # CIGAR offset + 4 bytes per CIGAR run out
    align_ms = float(np.mean([per_batch[e]["align_ms"] for e in args.edits]))
    n_per_launch = float(np.mean([b.n for b in batches]))
    bytes_per_pair = []
    for b, (s, st, off) in zip(batches, outs):
        runs = float(off[-1]) / b.n
        bytes_per_pair.append(float(b.pattern_lengths.mean() + b.text_lengths.mean()) + 8 + 4 + 1 + 8 + 4 * runs)
    bpp = float(np.mean(bytes_per_pair))
    hbm_gbs = float(peaks.get("hbm_gbs", PEAKS_FALLBACK["hbm_gbs"]))
    achieved_gbs = bpp * n_per_launch / (align_ms / 1000.0) / 1e9
    hbm_time_ms = bpp * n_per_launch / (hbm_gbs * 1e9) * 1000.0
    hbm = {"achieved": achieved_gbs, "peak": hbm_gbs, "unit": "GB/s", "frac": achieved_gbs / hbm_gbs,
           "time_ms": hbm_time_ms, "peak_source": peak_src}
    alu = None
    if cnt is not None:
        sm_max = float(peaks.get("sm_max_mhz", PEAKS_FALLBACK["sm_max_mhz"]))
        alu = integer_roofline(cnt, [b.n for b in batches], [per_batch[e]["align_ms"] for e in args.edits], sm_max)
    if alu is not None and alu["time_ms"] > hbm_time_ms:
        roof = dict(alu)
        roof["hbm"] = hbm
    else:
        roof = {"bound": "hbm", "achieved": achieved_gbs, "peak": hbm_gbs, "unit": "GB/s",
                "frac": achieved_gbs / hbm_gbs, "peak_source": peak_src}
        if alu is not None:
            roof["alu"] = alu
    roof["kernel"] = ("the short-read path: ordering pass (pack, score bound, sort in groups of 1,024) and lane-per-pair "
                      "kernel (wavefronts, backtrace), timed together by the call's events")
    roof["bytes_per_pair"] = bpp
    roof["avg_launch_ms"] = align_ms
    roof["traffic"] = None
    if kernel_sources_digest() == NCU_TRAFFIC["sha"] and all(e in NCU_TRAFFIC["bytes_per_pair"] for e in args.edits):
        roof["traffic"] = float(np.mean([NCU_TRAFFIC["bytes_per_pair"][e] * b.n for e, b in zip(args.edits, batches)]))
        roof["traffic_source"] = ("ncu dram bytes of 1M-pair launches of %s, scaled to the launch (device sources "
                                  "%s)" % (NCU_KERNEL, NCU_TRAFFIC["sha"]))

    # bounded samples of the other workloads the metric names: batched vs
    # plain on mixed lengths, and p50/p99 latency of the serving trace
    samples = {}
    if not args.no_samples:
        samples["mixed_lengths_sample"] = mixed_sample(args.mixed_pairs, steps=3, warmup=2)
        samples["serving_sample"] = serving_experiment(args.serving_requests, args.workers, burst=False, one=False,
                                                       plain=True)

    line = {
        "metric": METRIC, "value": value, "unit": "pairs/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": headline_config(args.pairs, world, args.edits),
        "roofline": roof,
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": "pairs/s", "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                "steps": e2e_steps,
                "inputs": "page-locked host buffers, sequences back to back (no offset arrays): streamed "
                          "chunk by chunk into a device ring on a copy stream; outputs copied back",
                "host_numa": numa,
                "clocks": e2e_clocks,
                "phase_ms_per_call": {k: round(float(np.mean([t[k] for t in e2e_phases[-2 * e2e_steps:]])), 3)
                                      for k in ("h2d_ms", "align_ms", "general_ms", "cigar_ms", "d2h_ms",
                                                "total_ms")} if e2e_phases else None},
        "aligned_bases_per_s": value * bases_per_step / pairs_per_step,
        "gpu_launches": launches,
        "clocks": clocks,
        "mode": "batched: default path, each batch's device work replayed from a CUDA graph",
        "vs_plain": {"batched_over_plain": value / other_modes["plain"]["pairs_per_s"],
                     "batched_over_eager": value / other_modes["eager"]["pairs_per_s"], **other_modes},
        **samples,
        "by_edit_rate": {"E=%d%%" % e: {"pairs_per_s_kernel_path": batches[i].n / (per_batch[e]["total_ms"] / 1000.0),
                                         "align_kernel_ms": per_batch[e]["align_ms"],
                                         "call_ms": per_batch[e]["total_ms"],
                                         "deferred_pairs": per_batch[e]["deferred"],
                                         "kernels_per_call": per_batch[e]["launches"],
                                         "short_variant": per_batch[e]["variant"],
                                         "mean_score": float(outs[i][0].mean())}
                         for i, e in enumerate(args.edits)},
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
