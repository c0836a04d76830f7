"""Benchmark: CLS random walks on one GB300 (or N, as independent history shards).

Workload (default): 3D box of side 10, Sigma = (0.1, 10), Lambda = (1, 0.1),
c = 0.99, cosine-law incidence on x = 0, 200 flux bins, 1e8 histories per GPU
per step, FP64, persistent history-based tracker.  One step = one pass of the
whole walk (source, flights, events, track-length tallies) over 1e8 histories;
`value` is histories/s over all ranks, device-timed with CUDA events.  The same
workload also runs with FP32 tracking / FP64 tallies, and both arms report the
figure of merit FOM = 1 / (sigma_rel(<phi>)^2 T).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun each rank takes its own disjoint history range (weak scaling).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "histories/s and FOM 1/(sigma^2 T) at equal sigma, FP32-batched vs FP64-plain on 1 GB300"
L2_FLUSH_BYTES = 512 << 20  # > 129 MB L2
BOX_WORKLOAD = "box L=10, Sigma=(0.1,10), Lambda=(1,0.1), c=0.99, cosine incidence, 200 bins"

# Work per event of the benchmark workloads' kernels, for the issue-rate
# roofline (152 SMs x 4 warp instructions per clock): warp instructions per
# event counted by ncu (smsp__inst_executed.sum / events, one pass) on the
# full-size launch of the current kernels (1e8 histories; the sweep's 256 x 1e7),
# updated with each capture of a changed kernel.  A small launch counts more
# per event: its heavy-tailed last histories run in nearly empty warps.
# FP64_FLOP_PER_EVENT: the same event's FP64 arithmetic evaluated directly in
# FP64 with FP64 elementary functions (ln, sin/cos, division, sqrt), counted by
# ncu (DADD + DMUL + 2 DFMA) on that direct evaluation; reported beside the
# roofline as FP64-equivalent TFLOP/s for context.  The kernel evaluates the
# elementary functions in the integer pipes and is bound by issue and latency,
# not by the FP64 pipe.
FP64_WARP_INST_PER_EVENT = 76.0
FP32_WARP_INST_PER_EVENT = 19.4
FP64_FLOP_PER_EVENT = 148.8
# The FP64 box kernel's FP64 pipe busy fraction (ncu sm__pipe_fp64_cycles_active,
# `--set full` of a 1e7-history launch): its second limit beside the issue rate.
FP64_PIPE_ACTIVE = 0.60
# The diffusive workload's FP32 kernels (500 bins: no difference array).
DIFFUSIVE_WARP_INST_PER_EVENT = {"history": 20.2, "event": 20.7}
# The batched sweep's FP32 kernel (history_kernel<float, 0, 1>, 256 cases x
# 1e7 histories in one launch, autotuned shape): warp instructions per event
# and DRAM bytes of one full-size replay, the same one-pass ncu capture.
BATCH_FP32_WARP_INST_PER_EVENT = 26.5
BATCH_FP32_DRAM_BYTES_PER_LAUNCH = 13265664
# DRAM bytes of that full-size FP64 launch (the same one-pass capture); None
# whenever the kernel has changed since the capture.
FP64_DRAM_BYTES_PER_LAUNCH = 882688
SM_COUNT = 152           # GB300
DFMA_PER_SM_CLK = 2      # ncu: sm__sass_thread_inst_executed_op_dfma_pred_on.sum.peak_sustained = 304 / 152 SMs
ISSUE_PER_SM_CLK = 4     # one warp instruction per scheduler per clock, 4 schedulers


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--histories", type=int, default=None, help="override histories per step (tests only)")
    ap.add_argument("--no-fp32", action="store_true", help="skip the FP32-tracking arm")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 arm (profiling only)")
    ap.add_argument("--no-projected", action="store_true",
                    help="skip the arms that walk the box by its x-marginal (geometry 13)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="box", choices=["box", "diffusive", "batch", "suite"],
                    help="box: L=10 box (default, the headline line); diffusive: L=100 box, c=0.999, "
                         "history vs event schedule; batch: 256-case sweep, FP64 plain vs FP32 batched; "
                         "suite: the paper's 54 benchmark configurations (Tables 3-8), FP64")
    return ap.parse_args()


# ------------------------------------------------------------ distributed
def dist_setup():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch.distributed as dist
        backend = "nccl"
        import torch
        if not torch.cuda.is_available():
            backend = "gloo"
        dist.init_process_group(backend=backend)
        pg = dist
    return rank, world, local, pg


def barrier(pg):
    if pg is not None:
        pg.barrier()


def max_over_ranks(pg, v: float) -> float:
    if pg is None:
        return v
    import torch
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi sampling during the timed region (every 200 ms)."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None
        self._summary = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        """Median SM clock under load and the throttle reasons seen; computed once."""
        if self._summary is None:
            self._summary = self._read()
        return self._summary

    def _read(self):
        if self.proc is None or not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9 and parts[1].isdigit():
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [int(r[1]) for r in rows]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        loaded = [s for s in sm if s > 0.5 * max(sm)] or sm
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": int(rows[0][2]), "reasons": reasons,
                "samples": len(rows), "power_w_max": max(float(r[3]) for r in rows if r[3].replace(".", "").isdigit())}


# ------------------------------------------------------------ oracle timing
def oracle_rate(params, seconds_target: float, cores: int, first: int = 0, detail: dict | None = None,
                n_fixed: int | None = None):
    """Time the FP64 oracle on a bounded sample of the workload over `cores` processes
    (n_fixed histories if given, else about seconds_target of work).  `detail`, if
    given, receives the single-process pilot's rate and the events per second of the
    sample."""
    import oracle
    case = oracle.Case(*params[:7], int(params[7]), int(params[8]))
    t0 = time.perf_counter()
    pilot = 2000
    oracle.run(case, 1, first, pilot)
    rate1 = pilot / (time.perf_counter() - t0)
    n = n_fixed or max(cores * 2048, int(rate1 * cores * seconds_target))
    t0 = time.perf_counter()
    raw = oracle.run_parallel(case, 1, first, n, workers=cores)
    dt = time.perf_counter() - t0
    if detail is not None:
        detail.update(single_process_histories_per_s=rate1, events_per_s=raw["n_events"] / dt)
    return n / dt, n, dt, raw["workers"]


def reference_arm(args, rank, world, pg):
    from paper_1708_00765_gb300 import workloads
    if rank != 0:
        barrier(pg)
        return
    params = workloads.BOX_L10
    cores = os.cpu_count() or 1
    rates = []
    detail = {}
    for i in range(args.warmup + args.steps):
        r, n, dt, used = oracle_rate(params, 4.0, cores, first=i * 10_000_000, detail=detail, n_fixed=args.histories)
        if i >= args.warmup:
            rates.append((r, n, dt))
    value = sum(r for r, _, _ in rates) / len(rates)
    n_mean = int(sum(n for _, n, _ in rates) / len(rates))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "histories/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(d for _, _, d in rates) / len(rates),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": BOX_WORKLOAD, "histories_per_step_per_gpu": n_mean, "schedule": "history",
                   "precision": "fp64", "sample": "a bounded sample of the workload per step, on the host cores"},
        "cpu_baseline": {"value": value, "unit": "histories/s", "cores": used, "kind": "oracle",
                         "sample": f"{n_mean} histories of the box L=10 workload per step",
                         "events_per_s": detail["events_per_s"],
                         "single_process_histories_per_s": detail["single_process_histories_per_s"]},
        "e2e": {"value": value, "unit": "histories/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    barrier(pg)


# ------------------------------------------------------------------ our arm
def timed_runs(prob, n, seed, steps, warmup, flush, torch, stream, first_base=0):
    """Device seconds of `steps` runs of n histories after `warmup` untimed ones."""
    times = []
    for i in range(warmup + steps):
        flush.zero_()
        if i == warmup:
            prob.reset()
            if first_base:
                prob.set_option("first_history", first_base)
        start = torch.cuda.Event(enable_timing=True)
        stop = torch.cuda.Event(enable_timing=True)
        start.record(stream)
        prob.run(n, seed, stream=stream)
        stop.record(stream)
        if i >= warmup:
            times.append((start, stop))
    torch.cuda.synchronize()
    return sum(a.elapsed_time(b) for a, b in times) * 1e-3


def diffusive_workload(args, rank, world, pg):
    """L=100 box, c=0.999, 500 bins, FP32 tracking: history vs event schedule."""
    import torch
    import paper_1708_00765_gb300 as cls
    from paper_1708_00765_gb300 import workloads
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    params = workloads.BOX_DIFFUSIVE
    n = args.histories or workloads.BOX_DIFFUSIVE_HISTORIES
    stream = torch.cuda.current_stream()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    out = {}
    sampler = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    with sampler:
        for sched in ("history", "event"):
            prob = cls.Problem(params)
            prob.set_option("precision", "fp32")
            prob.set_option("schedule", sched)
            dev = timed_runs(prob, n, 1, args.steps, args.warmup, flush, torch, stream,
                             first_base=rank * (args.warmup + args.steps) * n)
            tal = prob.tallies()
            dev = max_over_ranks(pg, dev)
            rel = tal["sigma_total_flux"] / tal["total_flux"]
            out[sched] = {"histories_per_s": world * args.steps * n / dev, "ms_per_step": 1e3 * dev / args.steps,
                          "events_per_s": world * tal["n_events"] / dev,
                          "events_per_history": tal["n_events"] / tal["n_histories"],
                          "max_events": tal["max_events"], "R": tal["R"], "total_flux": tal["total_flux"],
                          "fom_total_flux": 1.0 / (rel * rel * dev / world)}
            prob.close()
    clk_mhz = sampler.summary().get("sm_mhz") or 2070.0
    peak = SM_COUNT * ISSUE_PER_SM_CLK * clk_mhz * 1e6 / 1e12
    for sched, r in out.items():
        ev_s = r["events_per_s"] / world
        achieved = DIFFUSIVE_WARP_INST_PER_EVENT[sched] * ev_s / 1e12
        r["roofline"] = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Twarp-inst/s",
                         "frac": achieved / peak, "kernel": f"{sched}_kernel<float, 3, 0>",
                         "work": f"{DIFFUSIVE_WARP_INST_PER_EVENT[sched]} warp instructions/event",
                         "peak_from": f"{SM_COUNT} SM x {ISSUE_PER_SM_CLK} issue/clk x {clk_mhz} MHz"}
    if rank == 0:
        h = out["history"]
        print(json.dumps({
            "metric": METRIC, "value": h["histories_per_s"], "unit": "histories/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": h["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "diffusive box L=100, Sigma=(1,10), Lambda=(0.5,0.2), c=0.999, 500 bins, FP32 tracking",
                       "histories_per_step_per_gpu": n, "l2": "flushed between steps"},
            "clocks": sampler.summary(), "history": h, "event": out["event"],
            "event_over_history": out["event"]["histories_per_s"] / h["histories_per_s"]}), flush=True)


def batch_workload(args, rank, world, pg):
    """256-case sweep at 1e7 histories per case: FP64 plain (one launch per case, no
    graph, default launch shape) vs FP32 and FP64 batched (all cases in one
    persistent launch replayed from a CUDA graph, launch shape and schedule chosen
    by the autotuner), equal N per case."""
    import torch
    import paper_1708_00765_gb300 as cls
    from paper_1708_00765_gb300 import workloads
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    cases = workloads.batch_sweep(256, seed=7, nbins=100)
    n = args.histories or 10_000_000
    stream = torch.cuda.current_stream()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    sampler = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    t64 = t64b = None
    tal64 = []
    same = None
    with sampler:
        # FP64 plain: one handle and one launch per case
        plain = [] if args.no_fp64 else [cls.Problem(c) for c in cases]
        for p in plain:
            p.run(min(n, 20_000), 1, stream=stream)  # warm-up
            p.reset()
        torch.cuda.synchronize()
        if plain:
            flush.zero_()
            start = torch.cuda.Event(enable_timing=True)
            stop = torch.cuda.Event(enable_timing=True)
            start.record(stream)
            for p in plain:
                p.run(n, 1, stream=stream)
            stop.record(stream)
            torch.cuda.synchronize()
            t64 = max_over_ranks(pg, start.elapsed_time(stop) * 1e-3)
            tal64 = [p.tallies() for p in plain]
            for p in plain:
                p.close()
        arms = {}
        tuned = {}
        for prec in ("fp32",) if args.no_fp64 else ("fp32", "fp64"):
            b = cls.Problem(cases, batch=True)
            b.set_option("precision", prec)
            tuned[prec] = b.autotune(max(4096, min(n // 16, 262_144)), seed=3, stream=stream)
            # per-case schedules, kept only if a whole-batch pilot is faster with them
            # (profiling runs skip them: their pilots would precede the captured launch)
            if not args.no_fp64:
                per_case = b.autotune_cases(65_536, seed=3, stream=stream)
                tuned[prec]["event_schedule_cases"] = sum(1 for c in per_case if c == cls.CLS_SCHED_EVENT)
            dev = timed_runs(b, n, 1, args.steps, args.warmup, flush, torch, stream)
            arms[prec] = (max_over_ranks(pg, dev) / args.steps, [b.tallies(k) for k in range(len(cases))])
            b.close()
        # identical outcomes: both precisions walk the same histories (seed 11,
        # ids 0..n-1 of every case) once more, untimed, recording each history's
        # outcome (reflected / transmitted / absorbed / capped) on the device
        codes = {}
        for prec in () if args.no_fp64 else ("fp32", "fp64"):
            b = cls.Problem(cases, batch=True)
            b.set_option("precision", prec)
            b.autotune(max(4096, min(n // 16, 262_144)), seed=3, stream=stream)  # cached: the choice above
            codes[prec] = torch.empty(len(cases) * n, dtype=torch.uint8, device="cuda")
            b.record_outcomes(codes[prec].data_ptr(), codes[prec].numel())
            b.run(n, 11, stream=stream)
            torch.cuda.synchronize()
            b.close()
        if codes:
            same = (codes["fp32"] == codes["fp64"]).view(len(cases), n).sum(1, dtype=torch.int64).cpu().numpy() / n
        del codes
    t32, tal32 = arms["fp32"]
    events32 = sum(t["n_events"] for t in tal32) / args.steps  # per replay (tallies of the timed steps)
    clk_mhz = sampler.summary().get("sm_mhz") or 2070.0
    peak = SM_COUNT * ISSUE_PER_SM_CLK * clk_mhz * 1e6 / 1e12
    roofline = None
    if BATCH_FP32_WARP_INST_PER_EVENT is not None:
        achieved = BATCH_FP32_WARP_INST_PER_EVENT * events32 / t32 / 1e12
        roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Twarp-inst/s",
                    "frac": achieved / peak,
                    "traffic": BATCH_FP32_DRAM_BYTES_PER_LAUNCH if n == 10_000_000 else None,
                    "kernel": "history_kernel<float, 0, 1>",
                    "work": f"{BATCH_FP32_WARP_INST_PER_EVENT} warp instructions/event x {events32:.4g} events/replay",
                    "peak_from": f"{SM_COUNT} SM x {ISSUE_PER_SM_CLK} issue/clk x {clk_mhz} MHz (sampled)"}
    if rank == 0 and args.no_fp64:
        print(json.dumps({"profiling": "FP32 batched arm only", "fp32_batched": {
            "histories_per_s": world * len(cases) * n / t32, "s_per_replay": t32, "events_per_replay": events32,
            "autotuned": tuned["fp32"]}, "roofline": roofline, "clocks": sampler.summary()}), flush=True)
        return
    if rank == 0:
        t64b, tal64b = arms["fp64"]
        ratios = []
        zs = []
        for a, b in zip(tal64, tal32):
            s64 = a["sigma_total_flux"]
            s32 = b["sigma_total_flux"]
            if s64 > 0 and s32 > 0:
                # FOM = 1 / (sigma^2 T), sigma and T of the same histories: the
                # batched tallies hold the timed steps' histories (steps x n)
                ratios.append((s64 * s64 * t64) / (s32 * s32 * t32 * args.steps))
                zs.append((b["total_flux"] - a["total_flux"]) / math.hypot(s64, s32))
        ratios.sort()
        events64 = sum(a["n_events"] for a in tal64)
        print(json.dumps({
            "metric": METRIC, "value": world * len(cases) * n / t32, "unit": "histories/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t32, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "batched sweep, 256 cases (seed 7), 100 bins", "histories_per_case": n,
                       "l2": "flushed between steps"},
            "clocks": sampler.summary(),
            "fp32_batched": {"histories_per_s": world * len(cases) * n / t32, "s_per_replay": t32,
                             "events_per_replay": events32, "autotuned": tuned["fp32"]},
            "roofline": roofline,
            "fp64_batched": {"histories_per_s": world * len(cases) * n / t64b, "s_per_replay": t64b,
                             "autotuned": tuned["fp64"]},
            "fp64_plain": {"histories_per_s": world * len(cases) * n / t64, "s_total": t64,
                           "events_per_s": events64 / t64},
            "fom_ratio_fp32_batched_over_fp64_plain": {"median": ratios[len(ratios) // 2], "min": ratios[0],
                                                       "max": ratios[-1], "cases": len(ratios)},
            "fp32_vs_fp64_z": {"max_abs": max(abs(z) for z in zs), "rms": math.sqrt(sum(z * z for z in zs) / len(zs)),
                               "note": "same seed: correlated draws, so this z is conservative"},
            "fp32_fp64_identical_outcomes": {"median": float(sorted(same)[len(same) // 2]), "min": float(same.min()),
                                             "max": float(same.max()), "overall": float(same.mean()),
                                             "histories_per_case": n, "seed": 11},
        }), flush=True)


def suite_workload(args, rank, world, pg):
    """The paper's benchmark suite (Tables 1-2 materials; d = 1 slab, 2 extruded,
    3 box; suites I and II): each configuration walked in FP64 on the GPU, timed with
    CUDA events, next to the paper's published CPU rate 1e9 / t_tot (another machine:
    context only) and the printed CLS values."""
    import torch
    from fractions import Fraction
    import paper_1708_00765_gb300 as cls
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    n = args.histories or 100_000_000
    stream = torch.cuda.current_stream()
    here = os.path.join(ROOT, "tests", "golden")
    with open(os.path.join(here, "paper_cls_suite1.json")) as f:
        g1 = json.load(f)
    with open(os.path.join(here, "paper_cls_suite2.json")) as f:
        g2 = json.load(f)
    mats = g1["materials"]
    rows = [(1, r) for r in g1["rows"]] + [(2, r) for r in g2["rows"]]
    out = []
    tot_t = 0.0
    tot_h = 0
    sampler = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    with sampler:
        for suite, r in rows:
            sig = [float(Fraction(v)) for v in mats[r["case"][0]]["sigma"]]
            lam = [float(Fraction(v)) for v in mats[r["case"][0]]["lambda"]]
            c = [float(v) for v in mats[r["case"][1]]["c"]]
            geom = {1: 11, 2: 2, 3: 3}[r["d"]]
            prob = cls.Problem((sig[0], sig[1], lam[0], lam[1], c[0], c[1], 10.0, geom, 100))
            if suite == 2:
                prob.set_option("source", "volume")
            prob.run(min(n, 100_000), 99, stream=stream)  # warm-up
            prob.reset()
            start = torch.cuda.Event(enable_timing=True)
            stop = torch.cuda.Event(enable_timing=True)
            prob.set_option("first_history", rank * n)
            start.record(stream)
            prob.run(n, 2019, stream=stream)
            stop.record(stream)
            stop.synchronize()
            dt = max_over_ranks(pg, start.elapsed_time(stop) * 1e-3)
            t = prob.tallies()
            prob.close()
            N = t["n_histories"]
            z = {}
            if suite == 1:
                obs = {"R": (t["R"], t["sigma_R"]), "T": (t["T"], t["sigma_T"]),
                       "phi": (t["total_flux"], t["sigma_total_flux"])}
            else:
                pl = (t["nR"] + t["nT"]) / N
                obs = {"L": (pl / 2, math.sqrt(pl * (1 - pl) / (N - 1)) / 2),
                       "phi": (t["total_flux"], t["sigma_total_flux"])}
            for k, (v, sd) in obs.items():
                pv, psd = float(r[k][0]), float(r[k][1])
                z[k] = round((v - pv) / math.sqrt(sd * sd + psd * psd), 2)
            paper_rate = 1e9 / float(r["t_tot_s"])
            rate = world * n / dt
            out.append({"suite": "I" if suite == 1 else "II", "case": r["case"], "d": r["d"], "cite": r["cite"],
                        "histories_per_s": rate, "events_per_history": t["n_events"] / N,
                        "paper_cpu_histories_per_s": paper_rate, "speedup_vs_paper_cpu": rate / paper_rate,
                        "z_vs_paper": z})
            tot_t += dt
            tot_h += world * n
    if rank == 0:
        zs = [abs(v) for o in out for v in o["z_vs_paper"].values()]
        sp = sorted(o["speedup_vs_paper_cpu"] for o in out)
        print(json.dumps({
            "metric": METRIC, "value": tot_h / tot_t, "unit": "histories/s", "n_gpus": world, "steps": 1, "warmup": 1,
            "ms_per_step": 1e3 * tot_t, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": "paper benchmark suite: 3 cases x 3 sub-cases x d in {1,2,3} x suites I, II "
                                   "(Tables 1-8), L = 10, 100 bins, FP64 history tracker",
                       "histories_per_configuration": n, "configurations": len(out)},
            "clocks": sampler.summary(),
            "speedup_vs_paper_cpu": {"median": sp[len(sp) // 2], "min": sp[0], "max": sp[-1],
                                     "note": "paper: 1e9 / t_tot on a Xeon E5-2680 v2 cluster, cores not stated"},
            "z_vs_paper": {"max_abs": max(zs), "rms": math.sqrt(sum(v * v for v in zs) / len(zs))},
            "configurations": out}), flush=True)


def main():
    args = parse()
    rank, world, local, pg = dist_setup()
    if args.impl == "reference":
        reference_arm(args, rank, world, pg)
        return
    if args.workload != "box":
        import paper_1708_00765_gb300 as cls
        cls.load(build_if_missing=True)
        {"diffusive": diffusive_workload, "batch": batch_workload, "suite": suite_workload}[args.workload](
            args, rank, world, pg)
        barrier(pg)
        return
    import torch
    import paper_1708_00765_gb300 as cls
    from paper_1708_00765_gb300 import workloads
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device (the walk never runs on the CPU)")
    torch.cuda.set_device(local)
    cls.load(build_if_missing=True)
    params = workloads.BOX_L10
    n = args.histories or workloads.BOX_L10_HISTORIES
    seed = 1
    stream = torch.cuda.current_stream()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    results = {}
    arms = ([] if args.no_fp64 else ["fp64"]) + ([] if args.no_fp32 else ["fp32"])
    if not args.no_projected and not (args.no_fp64 or args.no_fp32):
        arms += ["fp64_x", "fp32_x"]
    clocks = None
    for arm in arms:
        prob = cls.Problem(workloads.BOX_L10_X if arm.endswith("_x") else params)
        prob.set_option("precision", arm[:4])
        # rank r walks its own history ids: warm-up runs come first, the timed runs follow
        base = rank * (args.warmup + args.steps) * n
        if base:
            prob.set_option("first_history", base)
        barrier(pg)
        torch.cuda.synchronize()
        sampler = ClockSampler(local)
        with sampler:
            times = []
            for i in range(args.warmup + args.steps):
                flush.zero_()
                if i == args.warmup:
                    prob.reset()
                    if base:
                        prob.set_option("first_history", base + args.warmup * n)
                    torch.cuda.synchronize()
                    barrier(pg)
                start = torch.cuda.Event(enable_timing=True)
                stop = torch.cuda.Event(enable_timing=True)
                start.record(stream)
                prob.run(n, seed, stream=stream)
                stop.record(stream)
                if i >= args.warmup:
                    times.append((start, stop))
            torch.cuda.synchronize()
            barrier(pg)
        dev_s = sum(a.elapsed_time(b) for a, b in times) * 1e-3
        if arm == "fp64":
            clocks = sampler.summary()
        else:
            sampler.summary()
        tal = prob.tallies()
        dev_max = max_over_ranks(pg, dev_s)
        hist = world * args.steps * n
        rel = tal["sigma_total_flux"] / tal["total_flux"]
        results[arm] = {
            "histories_per_s": hist / dev_max,
            "ms_per_step": 1e3 * dev_max / args.steps,
            "events_per_s": world * tal["n_events"] / dev_max,
            "collisions_per_s": world * tal["n_coll"] / dev_max,
            "events_per_history": tal["n_events"] / tal["n_histories"],
            "R": tal["R"], "T": tal["T"], "A": tal["A"], "total_flux": tal["total_flux"],
            "sigma_total_flux": tal["sigma_total_flux"],
            "fom_total_flux": 1.0 / (rel * rel * dev_max / world) if rel > 0 else None,
            "launch_ms": 1e3 * dev_s / args.steps,
            "events_per_launch": tal["n_events"] / args.steps,
        }
        # end to end through the C ABI: host-side run + tallies (D2H + FP64 normalisation) per step
        if arm == "fp64":
            e2e_steps = max(1, args.steps)
            barrier(pg)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(e2e_steps):
                prob.run(n, seed, stream=stream)
                prob.tallies()
            e2e_s = max_over_ranks(pg, time.perf_counter() - t0)
            nbatch = prob.get_option("nbatch")
            results["e2e"] = {"value": world * e2e_steps * n / e2e_s, "unit": "histories/s",
                              "h2d_bytes_per_step": 48,
                              "d2h_bytes_per_step": nbatch * int(params[8]) * 8 + 4 * 8 + 9 * 8}
        prob.close()

    clk_mhz = (clocks or {}).get("sm_mhz") or 2070.0
    if "fp64" in results:
        r = results["fp64"]
        ev_s = r["events_per_launch"] / (r["launch_ms"] * 1e-3)
        achieved = FP64_WARP_INST_PER_EVENT * ev_s / 1e12
        peak = SM_COUNT * ISSUE_PER_SM_CLK * clk_mhz * 1e6 / 1e12
        r["roofline"] = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Twarp-inst/s",
                         "frac": achieved / peak, "traffic": FP64_DRAM_BYTES_PER_LAUNCH,
                         "kernel": "history_kernel<double>",
                         "work": f"{FP64_WARP_INST_PER_EVENT} warp instructions/event x {r['events_per_launch']:.4g} events/launch",
                         "peak_from": f"{SM_COUNT} SM x {ISSUE_PER_SM_CLK} issue/clk x {clk_mhz} MHz (sampled)",
                         "fp64_equivalent_tflops": FP64_FLOP_PER_EVENT * ev_s / 1e12,
                         "fp64_peak_tflops": SM_COUNT * DFMA_PER_SM_CLK * 2 * clk_mhz * 1e6 / 1e12,
                         "fp64_pipe_active_ncu": FP64_PIPE_ACTIVE}
    if "fp32" in results:
        r = results["fp32"]
        achieved = FP32_WARP_INST_PER_EVENT * r["events_per_launch"] / (r["launch_ms"] * 1e-3) / 1e12
        peak = SM_COUNT * ISSUE_PER_SM_CLK * clk_mhz * 1e6 / 1e12
        r["roofline"] = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Twarp-inst/s",
                         "frac": achieved / peak, "kernel": "history_kernel<float>",
                         "work": f"{FP32_WARP_INST_PER_EVENT} warp instructions/event",
                         "peak_from": f"{SM_COUNT} SM x {ISSUE_PER_SM_CLK} issue/clk x {clk_mhz} MHz"}
    if rank == 0 and "fp64" not in results:
        print(json.dumps({"profiling_only": True, **results}), flush=True)
    elif rank == 0:
        r64 = results["fp64"]
        line = {
            "metric": METRIC, "value": r64["histories_per_s"], "unit": "histories/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": r64["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": BOX_WORKLOAD,
                       "histories_per_step_per_gpu": n, "schedule": "history", "precision": "fp64",
                       "l2": "flushed between steps (512 MB write)", "seed": seed},
            "clocks": clocks,
            "e2e": results["e2e"],
            "gpu_launches": args.steps,
            "roofline": r64["roofline"],
            "fp64": r64,
        }
        if "fp32" in results:
            r32 = results["fp32"]
            line["fp32"] = r32
            if r32["fom_total_flux"] and r64["fom_total_flux"]:
                line["fom_ratio_fp32_over_fp64"] = r32["fom_total_flux"] / r64["fom_total_flux"]
        for arm in ("fp64_x", "fp32_x"):
            if arm in results:
                rx = dict(results[arm])
                rx["note"] = "same box walked by its x-marginal (geometry 13): same law, fewer draws"
                line[arm] = rx
                line["fom_ratio_" + arm + "_over_fp64"] = rx["fom_total_flux"] / r64["fom_total_flux"]
        if not args.no_cpu_baseline and world == 1:
            detail = {}
            rate, ns, dt, used = oracle_rate(params, 10.0, os.cpu_count() or 1, first=10**12, detail=detail)
            line["cpu_baseline"] = {"value": rate, "unit": "histories/s", "cores": used, "kind": "oracle",
                                    "sample": f"{ns} histories of the same workload ({dt:.1f} s)",
                                    "events_per_s": detail["events_per_s"],
                                    "single_process_histories_per_s": detail["single_process_histories_per_s"],
                                    "full_workload_s_extrapolated": n / rate}
        print(json.dumps(line), flush=True)
    barrier(pg)
    if pg is not None:
        pg.destroy_process_group()


if __name__ == "__main__":
    main()
