"""Autotuner for the launch parameters of pf_loglik.

For a problem shape (network tier, species, particles, observation times) it
times pf_loglik on a sample of theta rows for each candidate block size (lanes
per filter: 64, 96, 128) and launch order, and keeps the fastest.  Results are
cached in a JSON file keyed by the shape, so a serving process tunes once.
Results never depend on these parameters, only the time does: the filters'
histories are exact integer work, and the weights' sum is taken in chunks of
32 particles in an order that does not depend on the block size.
"""
from __future__ import annotations

import json
import os
import time
from pathlib import Path

import numpy as np

from . import pf

DEFAULT_CACHE = Path(os.environ.get("PF1606_AUTOTUNE_CACHE",
                                    Path.home() / ".cache" / "pf1606" / "autotune.json"))
BLOCKS = (64, 96, 128)


def shape_key(net: dict, N: int, K: int, T: int) -> str:
    R, U = np.asarray(net["reactants"]).shape
    tier = 4 if R <= 4 else 8 if R <= 8 else 16 if R <= 16 else 32
    nb = 1 << int(np.ceil(np.log2(max(N, 1))))
    return f"R{tier}_U{U}_N{nb}_K{K}_T{T}"


def _time_call(fn, reps: int) -> float:
    import torch
    fn()
    torch.cuda.synchronize()
    best = float("inf")
    for _ in range(reps):
        t0 = time.perf_counter()
        fn()
        torch.cuda.synchronize()
        best = min(best, time.perf_counter() - t0)
    return best


def tune(net: dict, thetas, x0, obs_times, y, C, sigma, N: int, seed: int = 1, reps: int = 2,
         sample_filters: int = 4096, cache: Path | None = DEFAULT_CACHE) -> dict:
    """Time the candidates on a theta sample (device-resident) and cache the best."""
    import torch
    th = np.asarray(thetas, np.float64)
    T = np.asarray(y).shape[0]
    rows = max(1, min(len(th), sample_filters // max(T, 1)))
    dev = torch.device("cuda", torch.cuda.current_device())
    th_d = torch.from_numpy(np.ascontiguousarray(th[:rows])).to(dev)
    y_d = torch.from_numpy(np.ascontiguousarray(y, dtype=np.float64)).to(dev)
    timings = {}
    for B in BLOCKS:
        for sched in (pf.PF_SCHED_NATURAL, pf.PF_SCHED_HEAVY_FIRST):
            def call():
                pf.pf_loglik(net, th_d, x0, obs_times, y_d, C, sigma, N, seed, block_threads=B,
                             schedule=sched)
            timings[f"{B}:{sched}"] = _time_call(call, reps)
    best = min(timings, key=timings.get)
    B, sched = (int(v) for v in best.split(":"))
    result = {"block_threads": B, "schedule": sched, "timings_s": timings, "sample_rows": rows}
    if cache is not None:
        key = shape_key(net, N, len(obs_times), T)
        data = json.loads(cache.read_text()) if cache.exists() else {}
        data[key] = result
        cache.parent.mkdir(parents=True, exist_ok=True)
        cache.write_text(json.dumps(data, indent=1))
    return result


def lookup(net: dict, N: int, K: int, T: int, cache: Path = DEFAULT_CACHE) -> dict | None:
    """Cached choice for this shape, or None."""
    if not cache.exists():
        return None
    return json.loads(cache.read_text()).get(shape_key(net, N, K, T))


# --------------------------------------------------------------------------
# the batch engine's launch shape (pf_ctx_config)
# --------------------------------------------------------------------------
BATCH_BLOCKS = (64, 128)
BATCH_CLUSTERS = (2, 4)
BATCH_GRABS = (1, 4)


def split_rule(n_filters: int, sms: int = 152, blocks_per_sm: int = 4) -> bool:
    """A request is split over thread-block clusters when its filters alone
    cannot fill the GPU (fewer than one resident wave of blocks): its work then
    spreads over more SMs instead of ending the batch on a few of them.  A
    function of the request alone, so its results do not depend on the mix."""
    return n_filters < sms * blocks_per_sm


def mix_key(shapes) -> str:
    """Cache key of a request mix: the sorted (tier, N, K, T, split) shapes,
    theta counts rounded to powers of two."""
    items = sorted(shapes)
    return "mix:" + ";".join(",".join(str(v) for v in t) for t in items)


def tune_batch(make_requests, shapes, sample_frac: float = 0.125, cache: Path | None = DEFAULT_CACHE,
               n_slots: int = 1, max_particles: int = 4096, load_problems=None) -> dict:
    """Choose a context launch shape for a request mix by timing one batch of a
    sample of it per candidate (coordinate descent: threads per block for the
    small-network tier and for the others, then the cluster size of split
    requests, then the work-list grab).  make_requests(ctx, ids, frac) builds
    the sample's pf.Request list for a context whose problems load_problems(ctx)
    loaded; shapes identifies the mix in the cache."""
    key = mix_key(shapes)
    if cache is not None and cache.exists():
        hit = json.loads(cache.read_text()).get(key)
        if hit is not None:
            return hit
    has_split = any(t[-1] for t in shapes)

    def trial(cfg):
        ctx = pf.pf_ctx_create_config(0, n_slots, max_particles, **cfg)
        try:
            ids = load_problems(ctx)
            reqs = make_requests(ctx, ids, sample_frac, cfg["cluster_blocks"])
            pf.pf_ctx_run_batch(ctx, make_requests(ctx, ids, sample_frac / 8, cfg["cluster_blocks"]))
            t0 = time.perf_counter()
            pf.pf_ctx_run_batch(ctx, reqs)
            return time.perf_counter() - t0
        finally:
            pf.pf_ctx_destroy(ctx)

    best = {"block_threads": (128, 128, 128, 128), "cluster_blocks": 4, "grab": 1}
    timings = {}
    best_t = None
    for b_small in BATCH_BLOCKS:
        for b_large in BATCH_BLOCKS:
            cfg = dict(best, block_threads=(b_small, b_large, b_large, b_large))
            t = trial(cfg)
            timings[f"blocks {b_small}/{b_large}"] = t
            if best_t is None or t < best_t:
                best, best_t = cfg, t
    if has_split:
        for c in BATCH_CLUSTERS:
            if c == best["cluster_blocks"]:
                continue
            cfg = dict(best, cluster_blocks=c)
            t = trial(cfg)
            timings[f"cluster {c}"] = t
            if t < best_t:
                best, best_t = cfg, t
    for g in BATCH_GRABS:
        if g == best["grab"]:
            continue
        cfg = dict(best, grab=g)
        t = trial(cfg)
        timings[f"grab {g}"] = t
        if t < best_t:
            best, best_t = cfg, t
    result = dict(best, block_threads=list(best["block_threads"]), sample_s=best_t,
                  timings_s=timings, sample_frac=sample_frac)
    if cache is not None:
        data = json.loads(cache.read_text()) if cache.exists() else {}
        data[key] = result
        cache.parent.mkdir(parents=True, exist_ok=True)
        cache.write_text(json.dumps(data, indent=1))
    return result
