"""Drivers for the batching and serving patterns (measurement and examples).

run_hetero:  a heterogeneous set of requests evaluated (a) as one batch of the
             context (persistent kernels, one graph replay) and (b) as plain
             per-request pf_loglik launches, one after another.
run_serving: a Poisson stream of level-set batches served (a) by the context's
             continuous-batching worker (submit at arrival, several batches in
             flight) and (b) by a plain FIFO server that runs each request with
             its own pf_loglik launch.
Both check that the two arms give bit-identical log-likelihoods, and report
theta-likelihoods/s and latency percentiles.
"""
from __future__ import annotations

import threading
import time

import numpy as np

from . import pf
from . import workloads as W


def _load_problems(ctx, names):
    ids = {}
    for name in names:
        w = W.get(name)
        ids[name] = pf.pf_ctx_load_problem(ctx, w.net, len(w.prior_lo), w.x0, w.obs_times,
                                           w.observations(), w.C, w.sigma, model=w.model)
    return ids


def _plain(spec, w, cluster_blocks: int = 0):
    K = spec.K_use
    thr = spec.threshold if np.isfinite(spec.threshold) else None
    return pf.pf_loglik(w.net, spec.thetas, w.x0, w.obs_times[:K], w.observations()[:, :K, :],
                        w.C, w.sigma, spec.n_particles, spec.seed, reject_below=thr,
                        model=w.model, cluster_blocks=cluster_blocks)


def calibrate_thresholds(stream, rows: int = 256) -> dict:
    """Level-set threshold per network: the median log-likelihood (alpha = 50 %)
    of the first `rows` theta rows of that network's requests, evaluated fully
    once before the stream starts -- the sampler's quantile rule for epsilon_k."""
    out = {}
    for name in sorted({s.problem for s in stream}):
        specs = [s for s in stream if s.problem == name]
        th = np.concatenate([s.thetas for s in specs])[:rows]
        s0 = specs[0]
        w = W.get(name)
        K = s0.K_use
        r = pf.pf_loglik(w.net, th, w.x0, w.obs_times[:K], w.observations()[:, :K, :], w.C,
                         w.sigma, s0.n_particles, 12345)
        out[name] = float(np.median(r["loglik"]))
    for s in stream:
        s.threshold = out[s.problem]
    return out


def run_hetero(mix, n_slots: int = 3, repeats: int = 1, tune: bool = True,
               tune_cache=None, tune_frac: float = 1 / 32) -> dict:
    """The mix as one batch of a context (persistent kernels, one graph replay)
    against plain per-request pf_loglik launches.  Requests whose filters
    cannot fill the GPU alone (autotune.split_rule) run split over thread-block
    clusters in both arms, with the same cluster size; the context's launch
    shape comes from the batch autotuner on a sample of the mix (tune=True:
    tune_frac of every request's theta rows per candidate)."""
    from . import autotune
    names = sorted({s.problem for s in mix})
    wl = {n: W.get(n) for n in names}
    rows = sum(len(s.thetas) for s in mix)
    split = [autotune.split_rule(len(s.thetas) * wl[s.problem].T) for s in mix]

    def splits(cluster):
        # a request splits when it cannot fill the GPU and its share fits a cluster block
        return [sp and pf.split_fits(s.n_particles, cluster, wl[s.problem].U)
                for s, sp in zip(mix, split)]

    def make(ctx, ids, frac, cluster):
        out = []
        for s, sp in zip(mix, splits(cluster)):
            m = max(1, int(np.ceil(len(s.thetas) * frac)))
            out.append(pf.Request(ids[s.problem], s.thetas[:m], s.n_particles, s.seed,
                                  K_use=s.K_use, cluster_blocks=cluster if sp else 0))
        return out

    shapes = [(s.problem, 1 << int(np.ceil(np.log2(len(s.thetas)))), s.n_particles, s.K_use,
               bool(sp)) for s, sp in zip(mix, split)]
    if tune:
        cfg = autotune.tune_batch(make, shapes, sample_frac=tune_frac, cache=tune_cache,
                                  load_problems=lambda c: _load_problems(c, names))
    else:
        cfg = {"block_threads": [128] * 4, "cluster_blocks": 4, "grab": 1}
    C = int(cfg["cluster_blocks"])
    split = splits(C)
    ctx = pf.pf_ctx_create_config(0, n_slots, 4096, block_threads=tuple(cfg["block_threads"]),
                                  cluster_blocks=C, grab=int(cfg["grab"]))
    try:
        ids = _load_problems(ctx, names)
        # warm-up: one small request per problem
        pf.pf_ctx_run_batch(ctx, [pf.Request(ids[n], wl[n].thetas(1), 64, 1, K_use=2)
                                  for n in names])
        batched = []
        for _ in range(repeats):
            reqs = make(ctx, ids, 1.0, C)
            t0 = time.perf_counter()
            pf.pf_ctx_run_batch(ctx, reqs)
            batched.append(time.perf_counter() - t0)
        stats = pf.pf_ctx_stats(ctx)
    finally:
        pf.pf_ctx_destroy(ctx)
    _plain(mix[0], wl[mix[0].problem])  # warm-up
    t0 = time.perf_counter()
    plain = [_plain(s, wl[s.problem], C if sp else 0) for s, sp in zip(mix, split)]
    t_plain = time.perf_counter() - t0
    same = all(np.array_equal(r.loglik, p["loglik"]) for r, p in zip(reqs, plain))
    tb = float(np.min(batched))
    return {"requests": len(mix), "theta_rows": rows, "split_requests": int(sum(split)),
            "launch_shape": {k: cfg[k] for k in ("block_threads", "cluster_blocks", "grab")},
            "tuner_timings_s": cfg.get("timings_s"),
            "batched_s": tb, "plain_s": t_plain,
            "batched_theta_per_s": rows / tb, "plain_theta_per_s": rows / t_plain,
            "speedup": t_plain / tb, "identical_results": bool(same),
            "filters": int(stats["filters"] // (repeats + 1) if repeats else 0)}


def _percentiles(lat):
    lat = np.asarray(lat)
    return {"p50_ms": 1e3 * float(np.percentile(lat, 50)),
            "p99_ms": 1e3 * float(np.percentile(lat, 99)),
            "mean_ms": 1e3 * float(lat.mean()), "max_ms": 1e3 * float(lat.max())}


def serve_batched(stream, n_slots: int = 3, mem_budget: int = 0) -> dict:
    names = sorted({s.problem for s in stream})
    wl = {n: W.get(n) for n in names}
    ctx = pf.pf_ctx_create(mem_budget, n_slots, 4096)
    try:
        ids = _load_problems(ctx, names)
        pf.pf_ctx_run_batch(ctx, [pf.Request(ids[n], wl[n].thetas(1), 64, 1, K_use=2)
                                  for n in names])
        reqs = [pf.Request(ids[s.problem], s.thetas, s.n_particles, s.seed, K_use=s.K_use,
                           loglik_threshold=s.threshold) for s in stream]
        submit_clock = {}
        failed = []

        def submitter():
            t0 = time.perf_counter()
            try:
                for r, s in zip(reqs, stream):
                    dt = s.arrival_s - (time.perf_counter() - t0)
                    if dt > 0:
                        time.sleep(dt)
                    pf.pf_submit(ctx, r)
                    submit_clock[r.id] = time.perf_counter()
            except Exception as e:  # surfaced by the polling loop below
                failed.append(e)

        th = threading.Thread(target=submitter, daemon=True)
        th.start()
        lat = []
        finish = []
        for r in reqs:
            while r.id is None:
                if failed:
                    raise failed[0]
                time.sleep(0.0005)
            while not pf.pf_poll(ctx, r, wait_ms=50):
                pass
            lat.append(r.t_done - r.t_submit)
            finish.append(r.t_done)
        th.join()
        span = max(finish) - min(r.t_submit for r in reqs)
        stats = pf.pf_ctx_stats(ctx)
    finally:
        pf.pf_ctx_destroy(ctx)
    rows = sum(len(s.thetas) for s in stream)
    return {"theta_per_s": rows / span, "span_s": span, "batches": stats["batches"],
            **_percentiles(lat), "loglik": [r.loglik for r in reqs]}


def serve_plain(stream) -> dict:
    """FIFO server: each request runs as its own pf_loglik launch, in arrival
    order, as soon as the previous one finished."""
    wl = {n: W.get(n) for n in {s.problem for s in stream}}
    _plain(stream[0], wl[stream[0].problem])  # warm-up
    t0 = time.perf_counter()
    lat, outs = [], []
    for s in stream:
        now = time.perf_counter() - t0
        if s.arrival_s > now:
            time.sleep(s.arrival_s - now)
        outs.append(_plain(s, wl[s.problem])["loglik"])
        lat.append(time.perf_counter() - t0 - s.arrival_s)
    span = time.perf_counter() - t0 - stream[0].arrival_s
    rows = sum(len(s.thetas) for s in stream)
    return {"theta_per_s": rows / span, "span_s": span, **_percentiles(lat), "loglik": outs}


def run_serving(stream, n_slots: int = 3, thresholds: bool = True) -> dict:
    thr = calibrate_thresholds(stream) if thresholds else {}
    b = serve_batched(stream, n_slots)
    p = serve_plain(stream)
    lb, lp = b.pop("loglik"), p.pop("loglik")
    same = all(np.array_equal(x, y) for x, y in zip(lb, lp))
    rejected = int(sum(np.isneginf(x).sum() for x in lb))
    return {"requests": len(stream), "theta_rows": int(sum(len(s.thetas) for s in stream)),
            "thresholds": thr, "rejected_rows": rejected,
            "batched": b, "plain": p, "identical_results": bool(same)}
