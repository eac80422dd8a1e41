#!/usr/bin/env python3
"""Benchmark: particle-filter log-likelihoods of many theta on one GB300.

One *step* is one pf_loglik call over the whole gene-expression workload
(4096 theta x 10 trajectories x 1000 particles x 50 observation times,
2 species / 4 reactions), inputs resident in HBM.  Reported:
  value        theta-likelihoods/s (whole job, all ranks),
  ssa_events_per_s, e2e (through the C ABI with host buffers, copies timed),
  roofline     FP64 pipe of the filter kernel (the hot kernel),
  cpu_baseline the oracle on the host cores, on a bounded sample.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank evaluates its own theta batch (weak
scaling, no collective on the data path); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time
from pathlib import Path

import numpy as np

ROOT = Path(__file__).resolve().parent
sys.path.insert(0, str(ROOT))

from paper_1606_08281_gb300 import workloads as W  # noqa: E402

WORKLOAD = "gene_expression"
# Filters per launch split over thread-block clusters where that measured
# faster: launches whose time is set by a few filters (birth_death: 200
# filters for 152 SMs; lac_gfp: a few filters with billions of events).  The
# many-filter workloads fill the GPU with one block per filter.
CLUSTER_BLOCKS = {"birth_death": 4, "lac_gfp": 4}
L2_FLUSH_BYTES = 256 << 20          # > 129 MB L2
# FP64 roofline of the filter kernel.  Nominal GB300 FP64 rate 1.25 TFLOP/s
# at the 2070 MHz maximum SM clock over 152 SMs = 4 flops per SM per clock.
FP64_FLOPS_PER_SM_CLK = 4.0
N_SMS = 152
SM_MAX_MHZ = 2070.0
FP64_PEAK_TFLOPS = FP64_FLOPS_PER_SM_CLK * N_SMS * SM_MAX_MHZ * 1e6 / 1e12
# FP64 cost of the SSA event's variate and division, counted by ncu's FP64
# instruction counters on the pf_fp64_probe kernels (FMA = 2 flops):
#   the kernels' division (approximate-reciprocal seed, third-order Newton
#   step, residual-corrected quotient): 5 DFMA + 1 DMUL = 6 operations,
#   11 flops (the IEEE division would take 7 DFMA + 1 DMUL = 8, 15 flops);
#   exp(): 14 DFMA + 2 DADD = 16 operations, 30 flops;
#   the table-driven -log(u): 6 DFMA + 2 DMUL + 4 DADD = 12 operations, 18 flops.
# The Exp(1) variate is a 2048-layer ziggurat: one multiply when the fast path
# accepts; with probability P_WEDGE a wedge test (y: 2 operations; d and the two
# bounding lines: 3; exp() in the 0.62 % of wedge tests the lines leave open;
# a rejected attempt, half of them, costs one more multiply), with probability
# P_TAIL the tail (log + 1 add).  P_WEDGE + P_TAIL = 1 - mean of x_{i+1}/x_i
# over the layers = 0.003420; P_TAIL = (1/2048) / (r + 1).
FP64_OPS_DIV, FP64_FLOPS_DIV = 6.0, 11.0
FP64_OPS_EXP, FP64_FLOPS_EXP = 16.0, 30.0
FP64_OPS_LOG, FP64_FLOPS_LOG = 12.0, 18.0
P_TAIL = (1.0 / 2048) / (10.02289706840504086041 + 1.0)
P_WEDGE = 0.003420 - P_TAIL
P_WEDGE_OPEN = 0.0062
ZIG_OPS = 1.0 + P_WEDGE * (5.0 + P_WEDGE_OPEN * FP64_OPS_EXP + 0.5) + P_TAIL * (1.0 + FP64_OPS_LOG)
ZIG_FLOPS = 1.0 + P_WEDGE * (7.0 + P_WEDGE_OPEN * FP64_FLOPS_EXP + 0.5) + P_TAIL * (1.0 + FP64_FLOPS_LOG)


# DRAM bytes per launch of the filter kernel on the 4096-theta gene-expression
# workload: ncu dram__bytes_read.sum + dram__bytes_write.sum of the current
# kernel on its 152-theta case (229 120 + 0 bytes, one launch) scaled by the
# filters processed (x 4096/152).
FILTER_TRAFFIC_BYTES = 229_120 * 4096 / 152


def flops_per_event(R: int) -> float:
    """Algorithmic FP64 flops of one direct-method SSA event: R propensity
    products, R-1 prefix additions, u2*a0, t + tau, one Exp(1) variate
    (ziggurat, expected cost), one division."""
    return R + (R - 1) + 1.0 + 1.0 + ZIG_FLOPS + FP64_FLOPS_DIV


def ops_per_event(R: int) -> float:
    """The same work in FP64 pipe operations (each DFMA/DMUL/DADD = 1)."""
    return R + (R - 1) + 1.0 + 1.0 + ZIG_OPS + FP64_OPS_DIV


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples during the timed region (SM clock, reasons)."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.file = None

    def start(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.file, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.file.flush()
        self.file.seek(0)
        rows = [r.split(",") for r in self.file.read().strip().splitlines() if r.count(",") >= 8]
        os.unlink(self.file.name)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except ValueError:
                continue
            for name, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------ oracle leg
_ORACLE_CACHE = {}


def _oracle_warm(name):
    """Worker start-up: import the oracle and load the workload once."""
    sys.path.insert(0, str(ROOT))
    from oracle import pf_oracle
    if name not in _ORACLE_CACHE:
        w = W.get(name)
        _ORACLE_CACHE[name] = (pf_oracle, w, w.thetas(), w.observations())
    return os.getpid()


def _oracle_row(args):
    """Worker: the oracle on one theta row; returns its SSA event count."""
    name, m = args
    _oracle_warm(name)
    pf_oracle, w, th, y = _ORACLE_CACHE[name]
    r = pf_oracle.pf_loglik(w.net, th[m:m + 1], w.x0, w.obs_times, y, w.C, w.sigma, w.N,
                            w.filter_seed, theta_ids=[m], model=w.model)
    return int(r["events"][r["status"] == 0].sum())


def _windowed(warm, warm_arg, row, tasks, seconds: float):
    """Run `row` over `tasks` on one spawned single-threaded process per host
    core (each warmed up by `warm` before the clock starts) and count the rows
    finished within the wall-time window; the pool is terminated at its end,
    so a row that would run for long cannot hold the leg past the window.
    Returns (rows finished, sum of their row values, wall seconds, cores)."""
    import multiprocessing as mp
    cores = os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    pool = ctx.Pool(cores)
    done, total = 0, 0
    try:
        pool.map(warm, [warm_arg] * cores, chunksize=1)
        t0 = time.time()
        deadline = t0 + seconds
        it = pool.imap_unordered(row, tasks, chunksize=1)
        while True:
            remaining = deadline - time.time()
            if remaining <= 0:
                break
            try:
                v = it.next(timeout=remaining)
            except (mp.TimeoutError, StopIteration):
                break
            done += 1
            total += v
        wall = time.time() - t0
    finally:
        pool.terminate()
        pool.join()
    return done, total, wall, cores


def oracle_baseline(name: str, seconds: float) -> dict:
    """The filter oracle as it stands, one single-threaded process per host
    core, taking theta rows in row order (starting over when a short batch is
    exhausted before the window ends)."""
    w = W.get(name)
    n_tasks = max(w.M, 50_000)
    done, events, wall, cores = _windowed(_oracle_warm, name, _oracle_row,
                                          [(name, m % w.M) for m in range(n_tasks)], seconds)
    return {
        "value": done / wall if wall > 0 else 0.0,
        "unit": "theta-likelihoods/s",
        "cores": cores,
        "kind": "oracle",
        "ssa_events_per_s": events / wall if wall > 0 else 0.0,
        "sample": (f"{done} theta rows (x{w.T} trajectories x {w.N} particles x {w.K} times) of "
                   f"the {name} batch, taken in row order (cycling) by {cores} single-threaded "
                   f"oracle processes; rate = rows finished / wall time of the {wall:.1f} s "
                   f"window"),
        "wall_s": wall,
    }


def _exact_warm(key):
    """Worker start-up for the FSP / ODE oracle legs: key = (leg, workload, M)."""
    sys.path.insert(0, str(ROOT))
    if key not in _ORACLE_CACHE:
        leg, name, M = key
        if leg == "ode":
            from oracle import ode as mod
            w = W.erk()
            w.M = M
        else:
            from oracle import fsp as mod
            w = W.get(name)
        _ORACLE_CACHE[key] = (mod, w, w.thetas(), w.observations())
    return os.getpid()


def _exact_row(args):
    """Worker: the FSP or ODE oracle's log-likelihood of one theta row."""
    key, m = args
    _exact_warm(key)
    mod, w, th, y = _ORACLE_CACHE[key]
    if key[0] == "ode":
        mod.loglik(th[m], w.patterns, w.obs_times, y)
    else:
        for t in range(w.T):
            mod.loglik(w.net, th[m], w.x0, w.fsp_box, w.obs_times, y[t], w.C, w.sigma, w.model)
    return 0


def exact_baseline(leg: str, name: str, M: int, seconds: float) -> dict:
    """The FSP (scipy expm_multiply) or ODE (scipy DOP853, rtol 1e-11) oracle
    as it stands on the same theta batch, one single-threaded process per host
    core, rows in row order."""
    key = (leg, name, M)
    done, _, wall, cores = _windowed(_exact_warm, key, _exact_row,
                                     [(key, m) for m in range(M)], seconds)
    what = ("ODE oracle (scipy DOP853, rtol 1e-11)" if leg == "ode"
            else "FSP oracle (scipy expm_multiply)")
    return {
        "value": done / wall if wall > 0 else 0.0,
        "unit": "theta-likelihoods/s",
        "cores": cores,
        "kind": "oracle",
        "sample": (f"{done} theta rows of the {M}-row {name} batch, in row order, by {cores} "
                   f"single-threaded {what} processes; rate = rows finished / wall time of the "
                   f"{wall:.1f} s window"),
        "wall_s": wall,
    }


def run_reference_exact(a) -> None:
    """The reference arm of --mode fsp / ode: the FSP or ODE oracle as it
    stands on the GPU arm's theta batch, each step a bounded window."""
    if a.mode == "fsp":
        w = fsp_workload(a.workload)
        leg, name, metric, config = "fsp", w.name, "exact FSP theta-likelihoods/s", fsp_config(w)
    else:
        w = ode_workload(a.ode_theta)
        leg, name, metric, config = "ode", "erk", "ODE theta-likelihoods/s", ode_config(w)
    per_step = max(5.0, min(30.0, 150.0 / max(1, a.steps + a.warmup)))
    for _ in range(a.warmup):
        exact_baseline(leg, name, w.M, per_step / 4)
    vals, last = [], None
    for _ in range(a.steps):
        last = exact_baseline(leg, name, w.M, per_step)
        vals.append(last["value"])
    value = float(np.mean(vals))
    print(json.dumps({
        "impl": "reference", "metric": metric, "mode": a.mode, "value": value,
        "unit": "theta-likelihoods/s", "n_gpus": a.gpus, "steps": a.steps, "warmup": a.warmup,
        "ms_per_step": 1e3 * w.M / value if value > 0 else None, "ms_per_step_extrapolated": True,
        "higher_is_better": True, "dtype": "f64", "data": "synthetic", "config": config,
        "cpu_baseline": {k: last[k] for k in ("kind", "cores", "sample")} | {"value": value,
                                                                           "unit": last["unit"]},
        "e2e": {"value": value, "unit": "theta-likelihoods/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0}}), flush=True)


def run_reference(a, rank: int) -> None:
    if rank != 0:
        return
    if a.mode in ("fsp", "ode"):
        run_reference_exact(a)
        return
    w = W.get(a.workload)
    per_step = max(5.0, min(30.0, 150.0 / max(1, a.steps + a.warmup)))
    for _ in range(a.warmup):
        oracle_baseline(a.workload, per_step / 4)
    vals = []
    last = None
    for _ in range(a.steps):
        last = oracle_baseline(a.workload, per_step)
        vals.append(last["value"])
    value = float(np.mean(vals))
    line = {
        "impl": "reference",
        "metric": "theta-likelihoods/s", "value": value, "unit": "theta-likelihoods/s",
        "n_gpus": a.gpus, "steps": a.steps, "warmup": a.warmup,
        "ms_per_step": 1e3 * w.M / value if value > 0 else None,
        "ms_per_step_extrapolated": True,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": config_of(w),
        "cpu_baseline": {k: last[k] for k in ("kind", "cores", "sample")} | {"value": value,
                                                                           "unit": last["unit"]},
        "e2e": {"value": value, "unit": "theta-likelihoods/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
        "ssa_events_per_s": last["ssa_events_per_s"],
    }
    print(json.dumps(line), flush=True)


def fsp_workload(name: str):
    """The FSP mode's workload: telegraph or birth_death (the others have no box)."""
    return W.get(name if name in ("telegraph", "birth_death") else "telegraph")


def fsp_config(w) -> dict:
    return {"workload": f"{w.name}: FSP box {list(map(int, w.fsp_box))}, K={w.K} T={w.T} M={w.M}",
            "l2": "flushed between timed steps (256 MiB write)"}


def ode_workload(M: int):
    w = W.erk()
    w.M = M
    return w


def ode_config(w) -> dict:
    return {"workload": f"erk: {w.M} theta (within a factor e of theta_bar) x "
                        f"{len(w.patterns)} input patterns x {w.K} FRET readings",
            "rtol": 1e-10, "atol": 1e-13,
            "l2": "flushed between timed steps (256 MiB write)"}


def config_of(w) -> dict:
    return {"workload": f"{w.name}: U={w.U} R={w.R} P={w.P} K={w.K} T={w.T} M={w.M} N={w.N}",
            "M_theta": w.M, "T_trajectories": w.T, "K_times": w.K, "N_particles": w.N,
            "species": w.U, "reactions": w.R,
            "l2": "flushed between timed steps (256 MiB write)",
            "parallelism": "weak: one theta batch per GPU"}


# ---------------------------------------------------------------- GPU leg
def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=WORKLOAD, choices=sorted(W.WORKLOADS))
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--max-theta", type=int, default=0,
                    help="profiling case: only the first M' theta rows (not a bench line)")
    ap.add_argument("--no-probe", action="store_true")
    ap.add_argument("--no-phases", action="store_true",
                    help="skip the extra launch that measures the per-phase shares")
    ap.add_argument("--particles", type=int, default=0,
                    help="particles per filter instead of the workload's N (not the contract's "
                         "workload: e.g. a population beyond shared memory)")
    ap.add_argument("--probe-only", action="store_true",
                    help="run the FP64 cost probe alone and print it")
    ap.add_argument("--mode", default="step", choices=["step", "hetero", "serve", "fsp", "ode"],
                    help="step: the contract's timed step; hetero: one batch of a "
                         "heterogeneous request mix vs plain per-request launches; serve: a "
                         "Poisson request stream, continuous batching vs a plain FIFO server; "
                         "fsp: the exact FSP likelihood of a workload with an FSP box "
                         "(telegraph, birth_death); ode: the deterministic Erk-model likelihood")
    ap.add_argument("--ode-theta", type=int, default=4096,
                    help="--mode ode: theta rows per launch (the Erk batch size)")
    ap.add_argument("--hetero-requests", type=int, default=64)
    ap.add_argument("--hetero-cascade-theta", type=int, default=4096,
                    help="--mode hetero: largest theta count of a cascade request")
    ap.add_argument("--no-tune", action="store_true",
                    help="--mode hetero: the default launch shape instead of the batch autotuner's")
    ap.add_argument("--serve-seconds", type=float, default=10.0)
    ap.add_argument("--serve-rate", type=float, default=200.0)
    ap.add_argument("--cluster", type=int, default=-1,
                    help="split each filter over a thread-block cluster of this many blocks "
                         "(pf_options.cluster_blocks; 0 = one block per filter; default: the "
                         "measured choice for the workload, CLUSTER_BLOCKS)")
    ap.add_argument("--autotune", action="store_true",
                    help="tune block size and launch order on a theta sample before timing")
    a = ap.parse_args()
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local = int(os.environ.get("LOCAL_RANK", 0))
    if a.impl == "reference":
        run_reference(a, rank)
        return

    import torch
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    from paper_1606_08281_gb300 import build, pf
    if rank == 0:
        build.build()
    if world > 1:
        dist.barrier()
    pf.load()
    if a.probe_only:
        print(json.dumps(fp64_probe(pf)), flush=True)
        return
    if a.mode == "fsp":
        run_fsp(a, pf)
        return
    if a.mode == "ode":
        run_ode(a, pf)
        return
    if a.mode != "step":
        run_pattern(a)
        return

    from paper_1606_08281_gb300 import multi
    w = W.get(a.workload)
    if a.cluster < 0:
        a.cluster = CLUSTER_BLOCKS.get(a.workload, 0)
    if a.max_theta:
        w.M = min(w.M, a.max_theta)
    if a.particles:
        w.N = a.particles
    th_np = np.ascontiguousarray(multi.rank_thetas(w, rank)[: w.M])
    y_np = w.observations()
    th = torch.from_numpy(th_np).to(dev)
    yd = torch.from_numpy(y_np).to(dev)
    M, T = w.M, w.T
    out = {"loglik": torch.empty(M, dtype=torch.float64, device=dev),
           "status": torch.empty(M, dtype=torch.uint8, device=dev),
           "events": torch.empty((M, T), dtype=torch.int64, device=dev)}
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    launch = {"block_threads": 0, "schedule": pf.PF_SCHED_AUTO, "cluster_blocks": a.cluster}
    if a.autotune:
        from paper_1606_08281_gb300 import autotune
        tuned = autotune.tune(w.net, th_np, w.x0, w.obs_times, y_np, w.C, w.sigma, w.N,
                              sample_filters=20 * 608, cache=None)
        launch = {"block_threads": tuned["block_threads"], "schedule": tuned["schedule"],
                  "cluster_blocks": a.cluster}

    def step():
        pf.pf_loglik(w.net, th, w.x0, w.obs_times, yd, w.C, w.sigma, w.N, w.filter_seed,
                     out=out, stream=stream.cuda_stream, model=w.model, **launch)

    for _ in range(a.warmup):
        step()
    torch.cuda.synchronize()
    ev_step = int(out["events"][out["status"] == 0].sum().item())   # finished rows' reactions
    # rows may end with PF_ST_BUDGET (a prior draw whose reactions outrun the
    # event budget: likelihood 0); nothing else may fail
    budget_rows = int((out["status"] == pf.PF_ST_BUDGET).sum().item())
    assert int(((out["status"] != 0) & (out["status"] != pf.PF_ST_BUDGET)).sum().item()) == 0

    # FP64 cost probe: FMA peak and the price of log / division
    probe = None if a.no_probe else fp64_probe(pf)

    clocks = ClockSampler(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    times = []
    for _ in range(a.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    torch.cuda.synchronize()
    clk = clocks.stop()
    local_ms = float(np.mean(times))
    ms = multi.max_over_ranks(local_ms, dev)
    if world > 1:
        dist.barrier()

    # end to end through the C ABI with host (pinned) buffers
    th_pin = torch.from_numpy(th_np).pin_memory()
    y_pin = torch.from_numpy(y_np).pin_memory()
    ll_pin = torch.empty(M, dtype=torch.float64).pin_memory()
    st_pin = torch.empty(M, dtype=torch.uint8).pin_memory()
    host_out = {"loglik": ll_pin.numpy(), "status": st_pin.numpy()}
    e2e_times = []
    for _ in range(a.e2e_steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        pf.pf_loglik(w.net, th_pin.numpy(), w.x0, w.obs_times, y_pin.numpy(), w.C, w.sigma, w.N,
                     w.filter_seed, out=host_out, model=w.model, cluster_blocks=a.cluster)
        e2e_times.append(time.perf_counter() - t0)
    if e2e_times:
        assert np.array_equal(host_out["loglik"], out["loglik"].cpu().numpy())
    e2e_s = multi.max_over_ranks(float(np.mean(e2e_times)) if e2e_times else float("nan"), dev)

    # where a filter's time goes: one more launch with the per-phase clocks,
    # outside the timed region (one block per filter only)
    phases = None
    if a.cluster <= 1 and not a.no_phases:
        ph = pf.pf_loglik(w.net, th, w.x0, w.obs_times, yd, w.C, w.sigma, w.N, w.filter_seed,
                          stream=stream.cuda_stream, model=w.model, phase_cycles=True,
                          **{k: v for k, v in launch.items() if k != "cluster_blocks"})
        torch.cuda.synchronize()
        ok = (ph["status"] == 0).cpu().numpy()
        cyc = ph["phase_cycles"].cpu().numpy().astype(np.float64)[ok].sum(axis=(0, 1))
        tot = float(cyc.sum())
        phases = {"resample_gather": cyc[0] / tot, "simulation": cyc[1] / tot,
                  "weights_increment": cyc[2] / tot,
                  "how": "SM clock64 cycles of each filter block per phase (thread 0, phases end "
                         "at block barriers), summed over the finished filters of one extra launch"}

    cpu = None
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        cpu = oracle_baseline(a.workload, a.cpu_seconds)

    if rank == 0:
        fpe = flops_per_event(w.R)
        achieved = fpe * ev_step / (local_ms * 1e-3) / 1e12
        ops_rate = ops_per_event(w.R) * ev_step / (local_ms * 1e-3) / 1e12
        ops_peak = FP64_PEAK_TFLOPS / 2.0
        value = world * M / (ms * 1e-3)
        h2d = th_np.nbytes + y_np.nbytes + w.obs_times.nbytes
        d2h = M * 8 + M
        line = {
            "metric": "theta-likelihoods/s", "value": value, "unit": "theta-likelihoods/s",
            "n_gpus": world, "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_of(w), "launch": launch,
            "ssa_events_per_s": world * ev_step / (ms * 1e-3),
            "events_per_step": ev_step, "budget_rows": budget_rows,
            "clocks": clk,
            "e2e": {"value": world * M / e2e_s, "unit": "theta-likelihoods/s",
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": 2 * a.steps,
            "roofline": {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS,
                         "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS,
                         "traffic": FILTER_TRAFFIC_BYTES if w.name == WORKLOAD and w.M == 4096 else None,
                         "kernel": (f"filter_kernel_cluster (FP64 pipe; {a.cluster}-block clusters)"
                                    if a.cluster > 1 else "filter_kernel (FP64 pipe)"),
                         "flops_per_event": fpe,
                         "fp64_ops_per_event": ops_per_event(w.R),
                         "fp64_pipe_ops_frac": ops_rate / ops_peak,
                         "peak_source": "nominal GB300 FP64 1.25 TFLOP/s = 4 flops/SM/clk x "
                                        "152 SMs x 2070 MHz",
                         "kernel_ms": local_ms},
            "fp64_probe": probe,
            "phase_share": phases,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def run_pattern(a) -> None:
    """Batching / serving measurements (one JSON line each)."""
    from paper_1606_08281_gb300 import serving
    if a.mode == "hetero":
        mix = W.hetero_mix(n_requests=a.hetero_requests, max_theta_cascade=a.hetero_cascade_theta)
        res = serving.run_hetero(mix, repeats=1, tune=not a.no_tune)
        line = {"metric": "theta-likelihoods/s", "mode": "hetero-batch",
                "value": res["batched_theta_per_s"], "unit": "theta-likelihoods/s",
                "higher_is_better": True, "dtype": "f64", "data": "synthetic",
                "config": {"workload": f"heterogeneous mix: {a.hetero_requests} requests over "
                                       "birth_death / gene_expression / cascade, theta 1-4096 "
                                       f"(cascade 1-{a.hetero_cascade_theta}), N 256-4096, K 10-100 "
                                       "(seed 4001), plus one Lac-Gfp request (32 rows x 4 "
                                       "trajectories, N 200, K 29); requests that cannot fill the "
                                       "GPU alone split over clusters in both arms",
                           "launch_shape": "batch autotuner on a 1/32 sample" if not a.no_tune
                           else "defaults"},
                "plain_per_request": res["plain_theta_per_s"], **res}
    else:
        stream = W.serving_stream(rate_hz=a.serve_rate, duration_s=a.serve_seconds)
        res = serving.run_serving(stream)
        line = {"metric": "theta-likelihoods/s", "mode": "serving",
                "value": res["batched"]["theta_per_s"], "unit": "theta-likelihoods/s",
                "higher_is_better": True, "dtype": "f64", "data": "synthetic",
                "config": {"workload": f"Poisson {a.serve_rate:.0f}/s for {a.serve_seconds:.0f} s (seed 5001): "
                                       "gene_expression (theta 4-512, N 256, K 10) and cascade "
                                       "(theta 1-32, N 128, K 5), coin-flipped"},
                **res}
    print(json.dumps(line), flush=True)


def fsp_ops(w, th) -> float:
    """Algorithmic FP64 operations of the FSP uniformization for theta rows th:
    per row, lambda = max over the box of a_0(x); per interval, nsub sub-steps
    of jmax stencil products; each product costs R + 2 fused multiply-adds per
    state (R inflows from the predecessors, the diagonal term, the weighted
    sum of the series)."""
    box = np.asarray(w.fsp_box, np.int64)
    grids = np.meshgrid(*[np.arange(n + 1) for n in box], indexing="ij")
    X = np.stack([g.reshape(-1) for g in grids], axis=1)
    reac = np.asarray(w.net["reactants"], np.int64)
    h = np.ones((X.shape[0], reac.shape[0]))
    for r in range(reac.shape[0]):
        for u in range(reac.shape[1]):
            if reac[r, u] == 1:
                h[:, r] *= X[:, u]
            elif reac[r, u] == 2:
                h[:, r] *= X[:, u] * (X[:, u] - 1) / 2
    R, S = reac.shape[0], X.shape[0]
    dts = np.diff(np.concatenate([[0.0], w.obs_times]))
    total = 0.0
    for row in th:
        lam = float((h * row[:R][None, :]).sum(axis=1).max())
        for dt in dts:
            if dt <= 0 or lam <= 0:
                continue
            nsub = int(np.ceil(lam * dt / 1500.0))
            lh = lam * dt / nsub
            jmax = min(2047, int(np.ceil(lh + 8.5 * np.sqrt(lh) + 20.0)))
            total += nsub * jmax * S * (R + 2)
    return total


def run_fsp(a, pf) -> None:
    """The exact FSP likelihood of every theta row of a workload (one JSON line)."""
    import torch
    w = fsp_workload(a.workload)
    th_np = w.thetas()
    dev = torch.device("cuda", torch.cuda.current_device())
    th = torch.from_numpy(th_np).to(dev)
    yd = torch.from_numpy(w.observations()).to(dev)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def step():
        return pf.pf_fsp_loglik(w.net, th, w.x0, w.fsp_box, w.obs_times, yd, w.C, w.sigma,
                                model=w.model, stream=stream.cuda_stream)

    for _ in range(max(3, a.warmup)):
        r = step()
    torch.cuda.synchronize()
    assert int((r["status"] != 0).sum().item()) == 0
    clocks = ClockSampler(dev.index)
    clocks.start()
    times = []
    for _ in range(a.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    clk = clocks.stop()
    ms = float(np.mean(times))
    ops = fsp_ops(w, th_np)
    ops_rate = ops / (ms * 1e-3)
    peak_ops = FP64_PEAK_TFLOPS * 1e12 / 2.0          # one FP64 operation per lane per slot
    line = {"metric": "exact FSP theta-likelihoods/s", "mode": "fsp", "value": w.M / (ms * 1e-3),
            "unit": "theta-likelihoods/s", "n_gpus": 1, "steps": a.steps, "warmup": max(3, a.warmup),
            "ms_per_step": ms, "higher_is_better": True, "dtype": "f64", "data": "synthetic",
            "config": fsp_config(w),
            "clocks": clk,
            "roofline": {"bound": "alu", "achieved": ops_rate / 1e12, "peak": peak_ops / 1e12,
                         "unit": "T FP64 ops/s", "frac": ops_rate / peak_ops, "traffic": None,
                         "kernel": "fsp_kernel (FP64 pipe; the probability vectors stay in "
                                   "shared memory)",
                         "fp64_ops_per_step": ops},
            "cpu_baseline": (None if a.no_cpu_baseline
                             else exact_baseline("fsp", w.name, w.M, a.cpu_seconds))}
    print(json.dumps(line), flush=True)


# FP64 operations of one Dormand-Prince step of the Erk model: six new
# right-hand sides (per evaluation 56 multiplies/adds and 13 IEEE divisions at
# 8 operations each = 160), the stage combinations (stage s takes s - 1
# multiply-adds for the weighted sum and one for x + h (...): 2 + ... + 7 = 27
# per component) and the error estimate (6 multiply-adds, the step factor,
# the scale, one division and the square: ~20 per component).
ODE_OPS_PER_STEP = 6 * 160 + 14 * 27 + 14 * 20


def run_ode(a, pf) -> None:
    """The Erk-model likelihood of every theta row (one JSON line)."""
    import torch
    w = ode_workload(a.ode_theta)
    dev = torch.device("cuda", torch.cuda.current_device())
    th = torch.from_numpy(w.thetas()).to(dev)
    yd = torch.from_numpy(w.observations()).to(dev)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    out = None

    def step():
        return pf.pf_erk_loglik(th, w.patterns, w.obs_times, yd, diagnostics=True,
                                stream=stream.cuda_stream, out=out)

    for _ in range(max(3, a.warmup)):
        out = step()
    torch.cuda.synchronize()
    assert int((out["status"] != 0).sum().item()) == 0
    steps = int(out["steps"].to(torch.int64).sum().item())
    clocks = ClockSampler(dev.index)
    clocks.start()
    times = []
    for _ in range(a.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    clk = clocks.stop()
    ms = float(np.mean(times))
    ops_rate = steps * ODE_OPS_PER_STEP / (ms * 1e-3)
    peak_ops = FP64_PEAK_TFLOPS * 1e12 / 2.0
    line = {"metric": "ODE theta-likelihoods/s", "mode": "ode", "value": w.M / (ms * 1e-3),
            "unit": "theta-likelihoods/s", "n_gpus": 1, "steps": a.steps, "warmup": max(3, a.warmup),
            "ms_per_step": ms, "higher_is_better": True, "dtype": "f64", "data": "synthetic",
            "config": ode_config(w),
            "dp_steps_per_launch": steps, "clocks": clk,
            "roofline": {"bound": "alu", "achieved": ops_rate / 1e12, "peak": peak_ops / 1e12,
                         "unit": "T FP64 ops/s", "frac": ops_rate / peak_ops, "traffic": None,
                         "kernel": "erk_kernel (FP64 pipe; a lane pair per theta and pattern)",
                         "fp64_ops_per_dp_step": ODE_OPS_PER_STEP},
            "cpu_baseline": (None if a.no_cpu_baseline
                             else exact_baseline("ode", "erk", w.M, a.cpu_seconds))}
    print(json.dumps(line), flush=True)


def fp64_probe(pf) -> dict:
    blocks, threads = 152 * 4, 256
    res = {}
    iters = {0: 4096, 1: 256, 2: 512}
    iters[3] = 512
    iters[4] = 512
    iters[5] = 512
    for kind in (0, 1, 2, 3, 4, 5):
        pf.pf_fp64_probe(kind, blocks, threads, 16)          # warm-up
        ms, _ = pf.pf_fp64_probe(kind, blocks, threads, iters[kind])
        res[kind] = ms
    ops = blocks * threads * 8
    fma_rate = ops * iters[0] / (res[0] * 1e-3)            # FMA instructions per second
    log_rate = ops * iters[1] / (res[1] * 1e-3)            # log calls (+2 adds) per second
    div_rate = ops * iters[2] / (res[2] * 1e-3)
    mylog_rate = ops * iters[3] / (res[3] * 1e-3)
    exp_rate = ops * iters[4] / (res[4] * 1e-3)
    fdiv_rate = ops * iters[5] / (res[5] * 1e-3)
    return {
        "fast_div_per_s": fdiv_rate,
        "fast_div_fma_equiv_flops": 2 * fma_rate / fdiv_rate - 2.0,
        "exp_per_s": exp_rate,
        "exp_fma_equiv_flops": 2 * fma_rate / exp_rate - 2.0,
        "table_log_per_s": mylog_rate,
        "fma_tflops": 2 * fma_rate / 1e12,
        "log_per_s": log_rate, "div_per_s": div_rate,
        # cost of one call in FMA-equivalent flops (2 per FMA), minus its two adds
        "log_fma_equiv_flops": 2 * fma_rate / log_rate - 2.0,
        "div_fma_equiv_flops": 2 * fma_rate / div_rate - 2.0,
    }


if __name__ == "__main__":
    main()
