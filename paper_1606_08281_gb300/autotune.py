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
