"""Benchmark: CLS random walks on one GB300 (or N, as independent history shards).

Default workload (the headline line): the batched sweep of 256 cases (seed 7:
rods and 3D boxes, L in {0.1, 1, 10}, Sigma, Lambda log-uniform, c uniform;
100 flux bins) at 1e8 histories per case per step.  One step = one pass of the
whole walk (sources, flights, events, track-length tallies) over 2.56e10
histories: FP32 tracking with FP64 tallies, every case in one persistent
launch replayed from a CUDA graph.  `value` is histories/s over all ranks,
device-timed with CUDA events.  Against it, the same cases walked in FP64 one
launch per case (no graph, default launch shape): the figure of merit
FOM_X = 1 / (sigma_rel(X)^2 T) per case for X in {<phi>, R, T, worst bin},
the two arms' results in units of their combined standard error on
independent seeds, and the fraction of histories whose outcome is identical
on the same seed.  The same line carries the 3D box (L = 10, 1e8 histories
per step) in FP64 and FP32.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun each rank takes its own disjoint history range (weak scaling).
"""
from __future__ import annotations

import argparse
import csv
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
SWEEP_CASES, SWEEP_SEED, SWEEP_BINS = 256, 7, 100
SWEEP_HISTORIES = 100_000_000  # per case per step
SWEEP_WORKLOAD = ("batched sweep: 256 cases (seed 7; d in {rod, 3D box}, L in {0.1, 1, 10}, Sigma and Lambda "
                  "log-uniform, c uniform), 100 bins, FP32 tracking / exact tallies, the cases in one CUDA graph "
                  "replay (persistent launches as the autotuner groups them)")
BOX_WORKLOAD = "box L=10, Sigma=(0.1,10), Lambda=(1,0.1), c=0.99, cosine incidence, 200 bins"
SEED32, SEED64 = 1, 2   # the FP32 and FP64 arms draw from independent Philox keys
E2E_STEPS = 3           # end-to-end steps through the C ABI (host copies in the timed region)
ORACLE_HISTORIES = 1_000_000  # per case: the oracle's independent-seed check of the FP32 arm

SM_COUNT = 152           # GB300
ISSUE_PER_SM_CLK = 4     # one warp instruction per scheduler per clock, 4 schedulers
LANES = 32

# ------------------------------------------------------ algorithmic work model
# The work of Algorithm A per history, counted in thread operations (one
# 32-bit integer or FP32 operation, one FP32 approximate function, one shared
# atomic each), written from the algorithm -- not from the kernel -- and
# computed from each run's own counters (histories, events, collisions,
# absorptions, mean flight length):
#   draws: the source's (rod 1, slab and x-projected box 2, extruded 4, box 5),
#     two per event (collision and interface distances), one per collision
#     (scatter or absorb), one per rod / slab scatter or two per 3D scatter;
#   RNG: half a Philox4x32-10 block per draw (10 rounds of two 32x32->64
#     multiplies -- 4 operations -- and 4 XORs: 80 per block) plus 2 to form u;
#   per event: the two distances (2 logarithms at 2 operations, 2 scalings),
#     a boundary distance per tracked axis (3), the event select (5), the move
#     (1 per axis), the bin coordinates of the flight's ends (4), its end-bin
#     partials (2), one add per bin it touches (1 + E|omega_x| flight / dx),
#     and bookkeeping (2);
#   per collision the scatter test (1); per 3D scatter a new direction (mu,
#     sin theta, sin/cos phi, the three components and reciprocals: 8 + axes),
#     1 for the rod, 2 for the slab; per history the source (box 14, extruded
#     12, slab 3, rod 1) and the history-end statistics (6).
# Peak: every lane of every scheduler issuing one operation per clock,
# 152 SMs x 4 x 32 lanes x the sampled SM clock.
PHILOX_BLOCK_OPS = 80
UNIFORM_OPS = 2
# geometry -> (tracked axes, source draws, source ops, scatter draws, scatter ops, E|omega_x|)
GEOM_MODEL = {1: (1, 1, 1, 1, 1, 1.0), 2: (2, 4, 12, 2, 10, 0.5), 3: (3, 5, 14, 2, 11, 0.5),
              11: (1, 2, 3, 1, 2, 0.5), 13: (1, 2, 3, 1, 2, 0.5)}


def model_draws(geom: int, t: dict) -> float:
    """Random numbers Algorithm A draws for the histories of tallies `t` (suite I source)."""
    _, src_draws, _, sc_draws, _, _ = GEOM_MODEL[geom]
    return src_draws * t["n_histories"] + 2 * t["n_events"] + t["n_coll"] + sc_draws * (t["n_coll"] - t["nA"])


def algorithmic_ops(params, t: dict) -> float:
    """Thread operations of Algorithm A for the histories of tallies `t` of case `params`."""
    geom, L, nbins = int(params[7]), float(params[6]), int(params[8])
    axes, _, src_ops, _, sc_ops, wx = GEOM_MODEL[geom]
    N, ev, nc, na = t["n_histories"], t["n_events"], t["n_coll"], t["nA"]
    if ev == 0:
        return 0.0
    flight = t["total_flux"] * N / ev
    bins_touched = min(float(nbins), 1.0 + wx * flight / (L / nbins))
    per_event = 6 + 3 * axes + 5 + axes + 4 + 2 + bins_touched + 2
    return ((PHILOX_BLOCK_OPS / 2 + UNIFORM_OPS) * model_draws(geom, t) + per_event * ev + nc
            + sc_ops * (nc - na) + (src_ops + 6) * N)


def peak_ops(clk_mhz: float) -> float:
    return SM_COUNT * ISSUE_PER_SM_CLK * LANES * clk_mhz * 1e6


# --------------------------------------------- ncu counts of the current kernels
KERNEL_COUNTS = os.path.join(ROOT, "profiles", "kernel_counts.csv")


def kernel_counts(kernel: str, workload: str):
    """Events, warp and thread instructions and DRAM bytes of one launch of each kernel
    named in `kernel` ("a + b": summed), from the committed ncu summary of the
    current kernels (None when it lacks a row for one of them)."""
    if not os.path.exists(KERNEL_COUNTS):
        return None
    keys = ("events", "warp_inst", "thread_inst", "dram_read", "dram_write", "duration_ms")
    with open(KERNEL_COUNTS) as f:
        rows = list(csv.DictReader(line for line in f if not line.startswith("#")))
    out = dict.fromkeys(keys, 0.0)
    for k in (x.strip() for x in kernel.split("+")):
        row = next((r for r in rows if r["kernel"] == k and r["workload"] == workload), None)
        if row is None:
            return None
        for key in keys:
            out[key] += float(row[key])
    return out


def roofline(kernel, workload, ops_per_launch, launch_s, events_per_launch, clk_mhz, n_full: bool):
    """The bench's roofline object: algorithmic thread operations per launch over the
    launch's CUDA-event duration, against the issue peak; beside it, the kernel's own
    instruction count (ncu) as issue-slot occupancy, and its DRAM traffic."""
    achieved = ops_per_launch / launch_s
    peak = peak_ops(clk_mhz)
    out = {"bound": "alu", "achieved": achieved / 1e12, "peak": peak / 1e12, "unit": "Tthread-op/s",
           "frac": achieved / peak, "traffic": None, "kernel": kernel,
           "work": f"{ops_per_launch / events_per_launch:.1f} algorithmic thread operations/event x "
                   f"{events_per_launch:.4g} events/launch",
           "peak_from": f"{SM_COUNT} SM x {ISSUE_PER_SM_CLK} schedulers x {LANES} lanes x {clk_mhz} MHz (sampled)",
           "issue": None}
    kc = kernel_counts(kernel, workload)
    if kc is not None:
        per_event = kc["warp_inst"] / kc["events"]
        issue_peak = SM_COUNT * ISSUE_PER_SM_CLK * clk_mhz * 1e6
        # DRAM traffic scales with the launch only while it is the tallies' first touch: kept
        # for a launch of the captured size
        out["traffic"] = kc["dram_read"] + kc["dram_write"] if n_full else None
        out["issue"] = {"warp_inst_per_event": per_event,
                        "threads_per_warp_inst": kc["thread_inst"] / kc["warp_inst"],
                        "frac": per_event * events_per_launch / launch_s / issue_peak,
                        "source": os.path.relpath(KERNEL_COUNTS, ROOT)}
    return out


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--histories", type=int, default=None,
                    help="histories per step (per case for the sweep); tests and profiling only")
    ap.add_argument("--workload", default="default", choices=["default", "sweep", "box", "diffusive", "suite"],
                    help="default: the sweep's headline line plus the box arms; sweep / box: one of them alone; "
                         "diffusive: L=100 box, c=0.999, history vs event schedule; suite: the paper's 54 "
                         "benchmark configurations (Tables 3-8), FP64")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 arms (profiling only)")
    ap.add_argument("--no-fp32", action="store_true", help="box: skip the FP32 arm")
    ap.add_argument("--no-projected", action="store_true",
                    help="box: skip the arms that walk the box by its x-marginal (geometry 13)")
    ap.add_argument("--no-oracle", action="store_true", help="skip the oracle's check of the FP32 sweep")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--oracle-histories", type=int, default=ORACLE_HISTORIES)
    return ap.parse_args()


# ------------------------------------------------------------ distributed
def dist_setup():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch
        import torch.distributed as dist
        dist.init_process_group(backend="nccl" if torch.cuda.is_available() else "gloo")
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


def merge_clocks(samplers):
    """One clocks record over several sampled regions: the median of their medians,
    the union of their throttle reasons."""
    s = [x.summary() for x in samplers if x.summary().get("sm_mhz")]
    if not s:
        return samplers[0].summary()
    return {"sm_mhz": statistics.median(x["sm_mhz"] for x in s), "sm_max_mhz": s[0]["sm_max_mhz"],
            "reasons": sorted({r for x in s for r in x["reasons"]}), "samples": sum(x["samples"] for x in s),
            "power_w_max": max(x["power_w_max"] for x in s)}


# ------------------------------------------------------------ oracle timing
def sweep_cases():
    from paper_1708_00765_gb300 import workloads
    return workloads.batch_sweep(SWEEP_CASES, seed=SWEEP_SEED, nbins=SWEEP_BINS)


def oracle_cases(cases):
    import oracle
    return [oracle.Case(*c[:7], int(c[7]), int(c[8])) for c in cases]


def oracle_pool(cores):
    """The oracle's process pool: spawn-started, before this process touches the GPU."""
    import multiprocessing as mp
    import oracle
    oracle.build()
    return mp.get_context("spawn").Pool(cores)


def oracle_sweep(pool, cases, seed, first, n):
    """Oracle runs of histories [first, first + n) of every case (case k with Philox
    counter word 3 = k), one task per case; returns an AsyncResult of raw tallies."""
    import oracle
    from dataclasses import astuple
    args = [(astuple(c), seed, first, n, k) for k, c in enumerate(oracle_cases(cases))]
    order = sorted(range(len(args)), key=lambda k: -cases[k][6] * (1 + cases[k][4] + cases[k][5]))
    res = pool.map_async(oracle._run_case, [args[k] for k in order], chunksize=1)
    return res, order


def oracle_sweep_rate(pool, cases, cores, n_per_case=None, seconds_target=15.0, first=10**12):
    """Histories/s of the FP64 oracle on a bounded sample of the sweep: the first
    n_per_case ids of every case (sized from a pilot for about seconds_target of work
    when not given), over the spawn pool of `cores` processes."""
    if n_per_case is None:
        pilot_n = 5000
        t0 = time.perf_counter()
        res, _ = oracle_sweep(pool, cases, SEED64, first, pilot_n)
        res.get()
        pilot = time.perf_counter() - t0
        n_per_case = int(min(5_000_000, max(pilot_n, pilot_n * seconds_target / max(pilot, 1e-3))))
    sized = n_per_case is not None and seconds_target is None
    for attempt in range(3):
        t0 = time.perf_counter()
        res, _ = oracle_sweep(pool, cases, SEED64, first + (attempt + 1) * 10**9, n_per_case)
        raws = res.get()
        dt = time.perf_counter() - t0
        # the pilot's time is mostly fixed costs: grow the sample until it takes about the target
        if sized or dt >= 0.5 * seconds_target or n_per_case >= 5_000_000:
            break
        n_per_case = int(min(5_000_000, n_per_case * seconds_target / max(dt, 1e-3)))
    n = len(cases) * n_per_case
    return {"value": n / dt, "n_per_case": n_per_case, "seconds": dt, "cores": cores,
            "events_per_s": sum(r["n_events"] for r in raws) / dt}


def reference_arm(args, rank, world, pg):
    """The base contract's reference arm for this tier: the FP64 oracle, as it stands,
    on the host cores, each step a bounded sample of the headline workload."""
    if rank != 0:
        barrier(pg)
        return
    cases = sweep_cases()
    cores = os.cpu_count() or 1
    pool = oracle_pool(cores)
    n_case = args.histories
    rates = []
    for i in range(args.warmup + args.steps):
        r = oracle_sweep_rate(pool, cases, cores, n_per_case=n_case, seconds_target=None if n_case else 4.0,
                              first=i * 10**10)
        n_case = r["n_per_case"]  # the first step's size, for all steps
        if i >= args.warmup:
            rates.append(r)
    pool.close()
    pool.join()
    value = sum(r["value"] for r in rates) / len(rates)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "histories/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(r["seconds"] for r in rates) / len(rates),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": SWEEP_WORKLOAD, "cases": SWEEP_CASES, "histories_per_case_per_step": n_case,
                   "sample": "a bounded sample of the workload per step (the first ids of every case), "
                             "walked by the FP64 oracle on the host cores"},
        "cpu_baseline": {"value": value, "unit": "histories/s", "cores": rates[0]["cores"], "kind": "oracle",
                         "sample": f"{n_case} histories of each of the {SWEEP_CASES} sweep cases per step",
                         "events_per_s": sum(r["events_per_s"] for r in rates) / len(rates)},
        "e2e": {"value": value, "unit": "histories/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    barrier(pg)


# ------------------------------------------------------------------ helpers
def stats_of(v):
    v = sorted(float(x) for x in v)
    if not v:
        return None
    return {"median": v[len(v) // 2], "min": v[0], "max": v[-1], "cases": len(v)}


def rel_sigma(value, sigma):
    return sigma / abs(value) if value != 0 and sigma > 0 else None


def worst_bin_rel_sigma(t):
    phi, sd = np.asarray(t["flux"]), np.asarray(t["flux_sigma"])
    ok = (phi > 0) & (sd > 0)
    return float(np.max(sd[ok] / phi[ok])) if ok.any() else None


FOM_KEYS = (("total_flux", "sigma_total_flux"), ("R", "sigma_R"), ("T", "sigma_T"))


def fom_ratios(tal32, tal64, t32, t64):
    """Per case FOM_X(FP32 batched) / FOM_X(FP64 plain), FOM = 1 / (sigma_rel^2 T),
    for X in {<phi>, R, T, worst-bin phi}.  sigma^2 scales as 1/N, so the ratio at
    equal N is the ratio at equal sigma: the FP64 time to reach the FP32 arm's sigma
    over the FP32 time.  T is each arm's whole-sweep time."""
    out = {}
    for key, skey in FOM_KEYS + (("worst_bin", None),):
        r = []
        for a, b in zip(tal32, tal64):
            if key == "worst_bin":
                s32, s64 = worst_bin_rel_sigma(a), worst_bin_rel_sigma(b)
            else:
                s32, s64 = rel_sigma(a[key], a[skey]), rel_sigma(b[key], b[skey])
            if s32 and s64:
                r.append((s64 * s64 * t64) / (s32 * s32 * t32))
        out[key] = stats_of(r)
    return out


def count_z(ka: int, na: int, kb: int, nb: int):
    """Two runs' counts of one outcome (ka of na histories, kb of nb) compared by the
    exact conditional (Fisher) test: under equal rates, given k = ka + kb, ka is
    hypergeometric (k of the na + nb histories, na of them in run a).  The two-sided
    p-value is returned as the normal z of the same tail probability, signed as
    ka/na - kb/nb; for large counts it is the combined-variance z with the pooled
    proportion (Eq. combined_var).  None when neither run saw the outcome, or both
    saw it every time."""
    from scipy import stats
    k, m = ka + kb, na + nb
    if k == 0 or k == m:
        return None
    dist = stats.hypergeom(m, k, na)
    tail = dist.sf(ka - 1) if ka >= k * na / m else dist.cdf(ka)
    z = float(stats.norm.isf(min(1.0, 2.0 * tail) / 2.0))
    return z if ka / na >= kb / nb else -z


def z_scores(tal_a, tal_b, keys=("R", "T", "A", "total_flux")):
    """Per case and observable, the difference of two runs in units of its standard
    error: <phi> with each run's own error, (a - b) / sqrt(sigma_a^2 + sigma_b^2)
    (paper Eq. combined_var); the counts R, T, A by the exact conditional test
    (count_z), since a rare outcome may have a handful of counts, or none, in one run.
    Returns the summary and the largest |z| with its case and observable."""
    zs = []
    for case, (a, b) in enumerate(zip(tal_a, tal_b)):
        na, nb = int(a["n_histories"]), int(b["n_histories"])
        for k in keys:
            if k in ("R", "T", "A"):
                z = count_z(int(round(a[k] * na)), na, int(round(b[k] * nb)), nb)
            else:
                comb = math.hypot(a["sigma_" + k], b["sigma_" + k])
                z = (a[k] - b[k]) / comb if comb > 0 else None
            if z is not None:
                zs.append((z, case, k, a[k], b[k]))
    v = np.array([z[0] for z in zs])
    worst = max(zs, key=lambda z: abs(z[0]))
    return {"max_abs": float(np.max(np.abs(v))), "rms": float(np.sqrt(np.mean(v * v))),
            "above_4": int(np.sum(np.abs(v) > 4)), "n": int(v.size),
            "worst": {"case": worst[1], "observable": worst[2], "a": worst[3], "b": worst[4]}}


def oracle_tallies(raw, case):
    import oracle
    return oracle.finalize(raw, case)


def timed_pass(run, steps, warmup, flush, torch, stream, before_timed=None):
    """CUDA-event times (s) of `steps` calls of run() after `warmup` untimed ones, L2
    flushed before each; before_timed() runs once between the two phases."""
    times = []
    for i in range(warmup + steps):
        flush.zero_()
        if i == warmup:
            if before_timed:
                before_timed()
            torch.cuda.synchronize()
        start = torch.cuda.Event(enable_timing=True)
        stop = torch.cuda.Event(enable_timing=True)
        start.record(stream)
        run()
        stop.record(stream)
        if i >= warmup:
            times.append((start, stop))
    torch.cuda.synchronize()
    return [a.elapsed_time(b) * 1e-3 for a, b in times]


# ---------------------------------------------------------------- the sweep
def sweep_arms(args, rank, world, pg, local, pool):
    """The 256-case sweep: FP32 batched + graph (timed, steps x n per case), end to end
    through the C ABI, FP64 plain (one launch per case, one pass of n per case), the
    identical-outcome records and the oracle's independent check."""
    import torch
    import paper_1708_00765_gb300 as cls
    cases = sweep_cases()
    nc = len(cases)
    n = args.histories or SWEEP_HISTORIES
    stream = torch.cuda.current_stream()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    out = {}
    # the oracle's independent check of the FP32 arm starts first and overlaps the GPU work
    oracle_job = None
    if pool is not None and rank == 0 and not args.no_oracle:
        oracle_job = oracle_sweep(pool, cases, SEED64, 0, args.oracle_histories)

    # ---- FP32 batched: every case in one persistent launch, replayed from a graph
    b32 = cls.Problem(cases, batch=True)
    b32.set_option("precision", "fp32")
    tuned = b32.autotune(max(4096, min(n // 16, 262_144)), seed=3, stream=stream)
    base = rank * (args.warmup + args.steps + E2E_STEPS) * n
    if base:
        b32.set_option("first_history", base)

    def reset32():
        b32.reset()
        b32.set_option("first_history", base + args.warmup * n)

    barrier(pg)
    s32 = ClockSampler(local)
    with s32:
        times = timed_pass(lambda: b32.run(n, SEED32, stream=stream), args.steps, args.warmup, flush, torch, stream,
                           before_timed=reset32)
        barrier(pg)
    t32 = max_over_ranks(pg, sum(times))
    tal32 = [b32.tallies(k) for k in range(nc)]
    # end to end through the C ABI: each step's run (its work list copied from pinned
    # host memory) and every case's tallies (device-to-host copy, FP64 normalisation)
    barrier(pg)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(E2E_STEPS):
        b32.run(n, SEED32, stream=stream)
        for k in range(nc):
            b32.tallies(k)
    e2e_s = max_over_ranks(pg, time.perf_counter() - t0)
    b32.close()
    events32 = sum(t["n_events"] for t in tal32) / args.steps
    ops32 = sum(algorithmic_ops(c, t) for c, t in zip(cases, tal32)) / args.steps
    out["fp32_batched"] = {
        "histories_per_s": world * nc * n * args.steps / t32, "ms_per_step": 1e3 * t32 / args.steps,
        "events_per_s": world * events32 * args.steps / t32,
        "collisions_per_s": world * sum(t["n_coll"] for t in tal32) / t32,
        "events_per_history": events32 / (nc * n), "autotuned": tuned,
        "events_per_step_by_geometry": {int(g): sum(t["n_events"] for c, t in zip(cases, tal32) if int(c[7]) == g)
                                        / args.steps for g in sorted({int(c[7]) for c in cases})},
        "launch_ms": [1e3 * x for x in times], "ops_per_step": ops32, "events_per_step": events32}
    out["e2e"] = {"value": world * nc * n * E2E_STEPS / e2e_s, "unit": "histories/s", "steps": E2E_STEPS,
                  "h2d_bytes_per_step": nc * 40 + 24,
                  "d2h_bytes_per_step": nc * (64 * SWEEP_BINS * 8 + 4 * 8 + 9 * 8)}

    if not args.no_fp64:
        # ---- FP64 plain: one handle and one launch per case, default launch shape, no graph
        plain = [cls.Problem(c) for c in cases]
        for p in plain:
            p.run(20_000, 99, stream=stream)  # warm-up (module load, first launch)
            p.reset()
            if rank:
                p.set_option("first_history", rank * n)
        torch.cuda.synchronize()
        barrier(pg)
        s64 = ClockSampler(local)
        with s64:
            flush.zero_()
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in plain]
            for p, (a, b) in zip(plain, ev):
                a.record(stream)
                p.run(n, SEED64, stream=stream)
                b.record(stream)
            torch.cuda.synchronize()
            barrier(pg)
        t64 = max_over_ranks(pg, ev[0][0].elapsed_time(ev[-1][1]) * 1e-3)
        tal64 = [p.tallies() for p in plain]
        for p in plain:
            p.close()
        events64 = sum(t["n_events"] for t in tal64)
        ops64 = sum(algorithmic_ops(c, t) for c, t in zip(cases, tal64))
        out["fp64_plain"] = {"histories_per_s": world * nc * n / t64, "s_per_pass": t64,
                             "events_per_s": world * events64 / t64, "ops_per_pass": ops64,
                             "events_per_pass": events64}
        out["clocks64"] = s64
        out["fom"] = fom_ratios(tal32, tal64, t32, t64)
        # the FOM ratio's two factors: FP32 plain (one launch per case, as the FP64 arm)
        # isolates precision, FP32 batched over FP32 plain isolates batching
        plain32 = [cls.Problem(c) for c in cases]
        for p in plain32:
            p.set_option("precision", "fp32")
            p.run(20_000, 99, stream=stream)
            p.reset()
            p.set_option("first_history", base + (args.warmup + args.steps + E2E_STEPS) * n)
        torch.cuda.synchronize()
        barrier(pg)
        flush.zero_()
        a32, z32 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a32.record(stream)
        for p in plain32:
            p.run(n, SEED32, stream=stream)
        z32.record(stream)
        torch.cuda.synchronize()
        t32p = max_over_ranks(pg, a32.elapsed_time(z32) * 1e-3)
        tal32p = [p.tallies() for p in plain32]
        for p in plain32:
            p.close()
        out["fp32_plain"] = {"histories_per_s": world * nc * n / t32p, "s_per_pass": t32p,
                             "fom_batched_over_plain": fom_ratios(tal32, tal32p, t32, t32p)["total_flux"],
                             "fom_plain_fp32_over_fp64": fom_ratios(tal32p, tal64, t32p, t64)["total_flux"]}
        out["fp32_batching_by_size"] = batching_by_size(cases, (100_000, 1_000_000), flush, stream)
        out["z_fp32_vs_fp64"] = z_scores(tal32, tal64)
        # ---- identical outcomes: both precisions walk ids [0, n) of every case on the FP64
        # arm's seed once more, untimed, recording each history's outcome on the device
        codes = {}
        for prec in ("fp32", "fp64"):
            b = cls.Problem(cases, batch=True)  # default launch shape: results do not depend on it
            b.set_option("precision", prec)
            codes[prec] = torch.empty(nc * n, dtype=torch.uint8, device="cuda")
            b.record_outcomes(codes[prec].data_ptr(), codes[prec].numel())
            b.set_option("first_history", rank * n)
            b.run(n, SEED64, stream=stream)
            torch.cuda.synchronize()
            b.close()
        same = np.array([int((codes["fp32"][k * n:(k + 1) * n] == codes["fp64"][k * n:(k + 1) * n]).sum())
                         for k in range(nc)]) / n
        del codes
        torch.cuda.empty_cache()
        out["identical_outcomes"] = {"median": float(np.median(same)), "min": float(same.min()),
                                     "overall": float(same.mean()), "histories_per_case": n, "seed": SEED64}
    out["clocks32"] = s32
    if oracle_job is not None:
        res, order = oracle_job
        raws = res.get()
        ocs = oracle_cases(cases)
        tal_o = [None] * nc
        for k, raw in zip(order, raws):
            tal_o[k] = oracle_tallies(raw, ocs[k])
        # oracle results carry the library's key names for the z-scores
        out["z_fp32_vs_oracle"] = z_scores(tal32, tal_o)
        out["z_fp32_vs_oracle"]["oracle_histories_per_case"] = args.oracle_histories
    out["tal32"] = tal32
    return out


# ------------------------------------------------------------------ the box
def box_arms(args, rank, world, pg, local):
    """The 3D box of side 10 (1e8 histories per step) in FP64 and FP32, plus the same
    box walked by its x-marginal (geometry 13)."""
    import torch
    import paper_1708_00765_gb300 as cls
    from paper_1708_00765_gb300 import workloads
    n = args.histories or workloads.BOX_L10_HISTORIES
    stream = torch.cuda.current_stream()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    arms = ([] if args.no_fp64 else ["fp64"]) + ([] if args.no_fp32 else ["fp32"])
    if not args.no_projected and not (args.no_fp64 or args.no_fp32):
        arms += ["fp64_x", "fp32_x"]
    results = {}
    samplers = []
    for arm in arms:
        params = workloads.BOX_L10_X if arm.endswith("_x") else workloads.BOX_L10
        prob = cls.Problem(params)
        prob.set_option("precision", arm[:4])
        base = rank * (args.warmup + args.steps) * n

        def reset():
            prob.reset()
            prob.set_option("first_history", base + args.warmup * n)

        if base:
            prob.set_option("first_history", base)
        barrier(pg)
        sampler = ClockSampler(local)
        with sampler:
            times = timed_pass(lambda: prob.run(n, 1, stream=stream), args.steps, args.warmup, flush, torch, stream,
                               before_timed=reset)
            barrier(pg)
        samplers.append(sampler)
        tal = prob.tallies()
        prob.close()
        dev = max_over_ranks(pg, sum(times))
        rel = tal["sigma_total_flux"] / tal["total_flux"]
        ops = algorithmic_ops(params, tal) / args.steps
        ev = tal["n_events"] / args.steps
        results[arm] = {
            "histories_per_s": world * args.steps * n / dev, "ms_per_step": 1e3 * dev / args.steps,
            "events_per_s": world * tal["n_events"] / dev, "collisions_per_s": world * tal["n_coll"] / dev,
            "events_per_history": tal["n_events"] / tal["n_histories"],
            "R": tal["R"], "T": tal["T"], "A": tal["A"], "total_flux": tal["total_flux"],
            "sigma_total_flux": tal["sigma_total_flux"],
            "fom_total_flux": 1.0 / (rel * rel * dev / world) if rel > 0 else None,
            "ops_per_launch": ops, "events_per_launch": ev, "launch_s": dev / args.steps}
    clk = merge_clocks(samplers) if samplers else None
    clk_mhz = (clk or {}).get("sm_mhz") or 2070.0
    full = n == workloads.BOX_L10_HISTORIES
    names = {"fp64": ("history_kernel<double, 3, 0>", "box"), "fp32": ("history_kernel<float, 3, 0>", "box"),
             "fp64_x": ("history_kernel<double, 13, 0>", "box_x"), "fp32_x": ("history_kernel<float, 13, 0>", "box_x")}
    for arm, r in results.items():
        k, w = names[arm]
        r["roofline"] = roofline(k, w, r["ops_per_launch"], r["launch_s"], r["events_per_launch"], clk_mhz, full)
    if "fp64" in results:
        for arm in ("fp32", "fp64_x", "fp32_x"):
            if arm in results and results[arm]["fom_total_flux"]:
                results["fom_ratio_" + arm + "_over_fp64"] = results[arm]["fom_total_flux"] / results["fp64"]["fom_total_flux"]
    results["clocks"] = clk
    results["workload"] = BOX_WORKLOAD
    results["histories_per_step"] = n
    return results


def batching_by_size(cases, sizes, flush, stream):
    """Batching's gain at fewer histories per case, where per-launch overheads and
    tails weigh more: the sweep batched (autotuned for the size, graph replay) against
    one handle and one launch per case (default shape), FP32, median of 3 passes each."""
    import torch
    import paper_1708_00765_gb300 as cls
    out = {}
    for n in sizes:
        b = cls.Problem(cases, batch=True)
        b.set_option("precision", "fp32")
        tuned = b.autotune(max(4096, min(n // 16, 262_144)), seed=3, stream=stream)
        tb = sorted(timed_pass(lambda: b.run(n, 7, stream=stream), 3, 1, flush, torch, stream))[1]
        b.close()
        plain = [cls.Problem(c) for c in cases]
        for p in plain:
            p.set_option("precision", "fp32")

        def run_plain():
            for p in plain:
                p.run(n, 7, stream=stream)
        tp = sorted(timed_pass(run_plain, 3, 1, flush, torch, stream))[1]
        for p in plain:
            p.close()
        out[f"{n:.0e}".replace("+0", "")] = {"batched_histories_per_s": len(cases) * n / tb,
                                             "plain_histories_per_s": len(cases) * n / tp,
                                             "batched_over_plain": tp / tb, "autotuned": tuned}
    return out


# ------------------------------------------------------------- headline line
def headline(args, rank, world, pg, local):
    import torch
    import paper_1708_00765_gb300 as cls
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device (the walk never runs on the CPU)")
    cores = os.cpu_count() or 1
    # the oracle's pool is spawn-started before this process first touches the GPU
    pool = oracle_pool(cores) if rank == 0 and (not args.no_oracle or (world == 1 and not args.no_cpu_baseline)) \
        else None
    torch.cuda.set_device(local)
    cls.load(build_if_missing=True)
    n = args.histories or SWEEP_HISTORIES
    sw = sweep_arms(args, rank, world, pg, local, pool)
    box = box_arms(args, rank, world, pg, local) if args.workload == "default" else None
    if rank != 0:
        if pool is not None:
            pool.close()
        return
    cases = sweep_cases()
    clk = merge_clocks([sw["clocks32"]] + ([sw["clocks64"]] if "clocks64" in sw else []))
    clk_mhz = clk.get("sm_mhz") or 2070.0
    f32 = sw["fp32_batched"]
    # the sweep's DRAM traffic is its tallies' first touch (13 MB, in L2 afterwards), the same at any
    # histories per case: the ncu capture at 1e7 per case stands for the full launch
    full = True
    line = {
        "metric": METRIC, "value": f32["histories_per_s"], "unit": "histories/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": f32["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": SWEEP_WORKLOAD, "cases": len(cases), "histories_per_case_per_step": n,
                   "bins": SWEEP_BINS, "fp32_seed": SEED32, "fp64_seed": SEED64,
                   "l2": "flushed between steps (512 MB write)"},
        "clocks": clk,
        "e2e": sw["e2e"],
        "gpu_launches": args.steps * launches_per_replay(f32["autotuned"], cases),
        "roofline": roofline(sweep_kernels(f32["autotuned"]), "sweep", f32["ops_per_step"],
                             f32["ms_per_step"] * 1e-3, f32["events_per_step"], clk_mhz, full),
        "fp32_batched": {k: v for k, v in f32.items() if k not in ("ops_per_step",)},
    }
    if "fp64_plain" in sw:
        p64 = sw["fp64_plain"]
        line["fp64_plain"] = {
            "histories_per_s": p64["histories_per_s"], "s_per_pass": p64["s_per_pass"],
            "events_per_s": p64["events_per_s"], "launches": len(cases),
            "roofline": roofline("history_kernel<double, 1|3>", "sweep_plain", p64["ops_per_pass"], p64["s_per_pass"],
                                 p64["events_per_pass"], clk_mhz, False)}
        if "fp32_plain" in sw:
            line["fp32_plain"] = dict(sw["fp32_plain"], note=(
                "the same cases in FP32, one launch per case: FOM(FP32 batched)/FOM(FP64 plain) = "
                "batching (FP32 batched over FP32 plain) x precision (FP32 plain over FP64 plain)"))
            line["fp32_batching_by_size"] = dict(sw["fp32_batching_by_size"], note=(
                "the same comparison at 1e5 and 1e6 histories per case (rates, not FOM: equal N on both sides)"))
        line["fom_fp32_batched_over_fp64_plain"] = dict(sw["fom"], note=(
            "per case, FOM = 1/(sigma_rel^2 T) with T the arm's whole-sweep time; equal N is equal sigma "
            "(sigma^2 ~ 1/N), so this is also T64/T32 at equal sigma"))
        line["z_fp32_vs_fp64"] = dict(sw["z_fp32_vs_fp64"], note="independent Philox keys (seeds 1 and 2); "
                                                                  "R, T, A, <phi> of every case")
        line["identical_outcomes"] = sw["identical_outcomes"]
    if "z_fp32_vs_oracle" in sw:
        line["z_fp32_vs_oracle"] = dict(sw["z_fp32_vs_oracle"], note="FP64 oracle, independent seed, first ids "
                                                                      "of every case")
    if box is not None:
        line["box_L10"] = box
    if world == 1 and not args.no_cpu_baseline and pool is not None:
        cb = oracle_sweep_rate(pool, cases, cores)
        line["cpu_baseline"] = {"value": cb["value"], "unit": "histories/s", "cores": cb["cores"], "kind": "oracle",
                                "sample": f"{cb['n_per_case']} histories of each of the {len(cases)} sweep cases "
                                          f"({cb['seconds']:.1f} s)",
                                "events_per_s": cb["events_per_s"],
                                "full_workload_s_extrapolated": len(cases) * n / cb["value"]}
    if pool is not None:
        pool.close()
        pool.join()
    print(json.dumps(line), flush=True)


def launches_per_replay(tuned, cases) -> int:
    """Kernel launches in one replay of the sweep's graph: one per geometry when the
    autotuner groups the cases by geometry, else one mixed launch."""
    return len({int(c[7]) for c in cases}) if tuned.get("group_geometry", 0) else 1


def sweep_kernels(tuned) -> str:
    """The FP32 sweep's kernels: one mixed-geometry launch, or one per geometry (rods,
    boxes; their cases' short histories take the warp-summed-counters instance)."""
    if tuned.get("group_geometry", 0):
        return "history_kernel<float, 1, 1> + history_kernel<float, 3, 1>"
    return "history_kernel<float, 0, 1>"


def box_only(args, rank, world, pg, local):
    import torch
    import paper_1708_00765_gb300 as cls
    torch.cuda.set_device(local)
    cls.load(build_if_missing=True)
    box = box_arms(args, rank, world, pg, local)
    if rank == 0:
        print(json.dumps({"workload": BOX_WORKLOAD, **{k: v for k, v in box.items()}}), flush=True)


# -------------------------------------------------------------- diffusive box
def diffusive_workload(args, rank, world, pg, local):
    """L=100 box, c=0.999, 500 bins, FP32 tracking: history vs event schedule."""
    import torch
    import paper_1708_00765_gb300 as cls
    from paper_1708_00765_gb300 import workloads
    torch.cuda.set_device(local)
    cls.load(build_if_missing=True)
    params = workloads.BOX_DIFFUSIVE
    n = args.histories or workloads.BOX_DIFFUSIVE_HISTORIES
    stream = torch.cuda.current_stream()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    out = {}
    sampler = ClockSampler(local)
    with sampler:
        for sched in ("history", "event"):
            prob = cls.Problem(params)
            prob.set_option("precision", "fp32")
            prob.set_option("schedule", sched)
            base = rank * (args.warmup + args.steps) * n

            def reset():
                prob.reset()
                prob.set_option("first_history", base + args.warmup * n)

            times = timed_pass(lambda: prob.run(n, 1, stream=stream), args.steps, args.warmup, flush, torch, stream,
                               before_timed=reset)
            tal = prob.tallies()
            dev = max_over_ranks(pg, sum(times))
            rel = tal["sigma_total_flux"] / tal["total_flux"]
            out[sched] = {"histories_per_s": world * args.steps * n / dev, "ms_per_step": 1e3 * dev / args.steps,
                          "events_per_s": world * tal["n_events"] / dev,
                          "events_per_history": tal["n_events"] / tal["n_histories"],
                          "max_events": tal["max_events"], "R": tal["R"], "total_flux": tal["total_flux"],
                          "fom_total_flux": 1.0 / (rel * rel * dev / world),
                          "ops_per_launch": algorithmic_ops(params, tal) / args.steps,
                          "events_per_launch": tal["n_events"] / args.steps, "launch_s": dev / args.steps}
            prob.close()
    clk_mhz = sampler.summary().get("sm_mhz") or 2070.0
    full = n == workloads.BOX_DIFFUSIVE_HISTORIES
    for sched, r in out.items():
        r["roofline"] = roofline("history_kernel<float, 3, 0>" if sched == "history" else "event_kernel<float, 3>",
                                 "diffusive", r["ops_per_launch"], r["launch_s"],
                                 r["events_per_launch"], clk_mhz, full)
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


# ------------------------------------------------------------- paper's suite
def suite_workload(args, rank, world, pg, local):
    """The paper's benchmark suite (Tables 1-2 materials; d = 1 slab, 2 extruded,
    3 box; suites I and II): each configuration walked in FP64 on the GPU, timed with
    CUDA events, next to the paper's published CPU rate 1e9 / t_tot (another machine:
    context only) and the printed CLS values."""
    import torch
    from fractions import Fraction
    import paper_1708_00765_gb300 as cls
    torch.cuda.set_device(local)
    cls.load(build_if_missing=True)
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
    sampler = ClockSampler(local)
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
    elif args.workload in ("default", "sweep"):
        headline(args, rank, world, pg, local)
        barrier(pg)
    else:
        {"box": box_only, "diffusive": diffusive_workload, "suite": suite_workload}[args.workload](
            args, rank, world, pg, local)
        barrier(pg)
    if pg is not None:
        pg.destroy_process_group()


if __name__ == "__main__":
    main()
