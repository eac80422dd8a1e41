"""Parallel runs of the filter oracle (test infrastructure only).

The oracle itself stays single-threaded; large parity checks split their
filters into independent tasks (theta rows and trajectories, each with its
own theta and trajectory ids in the random-number counter) and run them in
spawned processes, one per host core.  Processes are spawned, never forked,
so that a caller that has already initialised CUDA can use the pool.
"""
from __future__ import annotations

import multiprocessing as mp
import os

import numpy as np


def _run(task: dict) -> dict:
    from oracle import pf_oracle
    return pf_oracle.pf_loglik(**task)


def map_loglik(tasks: list[dict], processes: int | None = None) -> list[dict]:
    """pf_oracle.pf_loglik(**task) for every task, in order."""
    if not tasks:
        return []
    n = min(len(tasks), processes or os.cpu_count() or 1)
    if n == 1:
        return [_run(t) for t in tasks]
    ctx = mp.get_context("spawn")
    with ctx.Pool(n) as pool:
        return pool.map(_run, tasks, chunksize=1)


def filter_tasks(net, thetas, theta_ids, x0, obs_times, y, C, sigma, N, seed, *,
                 traj_ids=None, split_trajectories: bool = False, rows_per_task: int = 1,
                 budget: int | None = None, model=None, want_final_states: bool = False):
    """Tasks for map_loglik covering rows `theta_ids` (global ids of the rows
    of `thetas`) and the trajectories of y (ids traj_ids, default 0..T-1):
    rows_per_task rows per task, each trajectory a task of its own when
    split_trajectories.  Returns (tasks, where): where[i] = (row slice,
    trajectory slice) of task i in the full [M][T] result."""
    thetas = np.asarray(thetas, np.float64)
    theta_ids = np.asarray(theta_ids, np.int64)
    y = np.asarray(y, np.float64)
    T = y.shape[0]
    traj_ids = np.arange(T) if traj_ids is None else np.asarray(traj_ids, np.int64)
    tasks, where = [], []
    for r0 in range(0, len(thetas), rows_per_task):
        rs = slice(r0, min(len(thetas), r0 + rows_per_task))
        tsl = [slice(t, t + 1) for t in range(T)] if split_trajectories else [slice(0, T)]
        for ts in tsl:
            task = dict(net=net, thetas=thetas[rs], x0=x0, obs_times=obs_times, y=y[ts], C=C,
                        sigma=sigma, n_particles=N, seed=seed, theta_ids=theta_ids[rs],
                        traj_ids=traj_ids[ts], model=model, want_final_states=want_final_states)
            if budget is not None:
                task["budget"] = budget
            tasks.append(task)
            where.append((rs, ts))
    return tasks, where


def assemble(results: list[dict], where: list, M: int, T: int) -> dict:
    """Per-filter oracle outputs [M][T] from map_loglik results of
    filter_tasks.  loglik[m] is the sum over trajectories in order, -inf if
    any trajectory failed (the oracle's own rule)."""
    ll = np.zeros((M, T))
    st = np.zeros((M, T), np.uint8)
    ev = np.zeros((M, T), np.uint64)
    dg = np.zeros((M, T), np.uint64)
    fs = None
    for r, (rs, ts) in zip(results, where):
        ll[rs, ts] = r["ll_traj"]
        ev[rs, ts] = r["events"]
        dg[rs, ts] = r["digest"]
        # a per-trajectory status: the oracle's row status applies to every
        # trajectory of the task (one trajectory per task when split)
        st[rs, ts] = np.asarray(r["status"])[:, None]
        if "final_states" in r:
            if fs is None:
                fs = np.zeros((M, T) + r["final_states"].shape[2:], np.int32)
            fs[rs, ts] = r["final_states"]
    loglik = np.zeros(M)
    status = np.zeros(M, np.uint8)
    for m in range(M):
        s = 0.0
        for t in range(T):
            s = s + ll[m, t]
        bad = st[m][st[m] != 0]
        status[m] = bad[0] if len(bad) else 0
        loglik[m] = s if status[m] == 0 else -np.inf
    out = {"ll_traj": ll, "status_traj": st, "events": ev, "digest": dg, "loglik": loglik,
           "status": status}
    if fs is not None:
        out["final_states"] = fs
    return out


def _paths_rows(task: dict) -> np.ndarray:
    """Events fired by one unconditioned direct-method path per theta row."""
    from oracle import pf_oracle
    out = np.zeros(len(task["thetas"]), np.uint64)
    for i, th in enumerate(task["thetas"]):
        _, fired, _ = pf_oracle.ssa_paths(task["net"], th, task["x0"], task["times"], 1,
                                          seed=task["seed"], budget=task.get("budget", 1 << 20),
                                          rate_coef=task.get("rate_coef"))
        out[i] = fired[0]
    return out


def path_events(net, thetas, x0, times, seed: int, rows_per_task: int = 256,
                processes: int | None = None, rate_coef=None) -> np.ndarray:
    """Events of one oracle SSA path per theta row over `times` (a cost
    ranking of the rows for choosing test cases; not a filter result).
    rate_coef [R][d] composes the rates as in the model extensions."""
    thetas = np.asarray(thetas, np.float64)
    tasks = [dict(net=net, thetas=thetas[i:i + rows_per_task], x0=x0, times=times, seed=seed,
                  rate_coef=rate_coef)
             for i in range(0, len(thetas), rows_per_task)]
    n = min(len(tasks), processes or os.cpu_count() or 1)
    if n <= 1:
        parts = [_paths_rows(t) for t in tasks]
    else:
        with mp.get_context("spawn").Pool(n) as pool:
            parts = pool.map(_paths_rows, tasks, chunksize=1)
    return np.concatenate(parts) if parts else np.zeros(0, np.uint64)
