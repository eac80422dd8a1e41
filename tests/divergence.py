"""First-divergence harness: where and why another implementation's filter
leaves the oracle's (test infrastructure).

For one filter (theta row with its id, trajectory with its id) whose GPU
result differs from the oracle's, trace_filter

  1. finds the first interval k* after which the two disagree, by bisection
     over the number of observation times (a filter run on the first K'
     times follows exactly the first K' intervals of the full filter: the
     random-number counters do not depend on K);
  2. lists the particle slots whose states after interval k* differ;
  3. tries the two admissible explanations, both last-place effects of a
     logarithm or exponential implemented differently on the two sides:
       * an integer resampling weight off by one: a weight of interval k*-1
         whose real value 2^32 exp(e_i - max e) lies within 2^-20 of an
         integer (two units in the last place of exp) is moved by one in that
         direction, the ancestors are drawn again with the oracle's
         systematic resampling, and every particle of interval k* is
         replayed; the explanation holds if all end states then equal the
         GPU's;
       * one direct-method draw: each mismatching particle is replayed by the
         oracle draw by draw, and at every fragile draw -- a wedge test within
         4 ulps of exp(-x), a tail variate r - log(u), a time test within 4 ulps
         of t_k, a selection within 4 ulps of a prefix sum -- the other branch
         (or E one ulp up or down) is taken; the explanation holds if the
         replay then ends in the GPU's state;
  4. reports (k*, the particles, the explanation) and whether every
     mismatching particle is explained ("traced").

A mismatch that no such last-place alternative explains is a real
difference between the implementations, and the parity tests fail on it.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from oracle import pf_oracle

FRAGILE_ULPS = 4.0
ALT_TIME_FLIP, ALT_CHOSEN_UP, ALT_CHOSEN_DOWN, ALT_WEDGE_FLIP = 1, 2, 3, 4
ALT_E_UP, ALT_E_DOWN = 5, 6
RP_WEDGE, RP_TAIL = 1, 2


@dataclass
class Report:
    traced: bool
    k: int | None = None
    particles: list = field(default_factory=list)   # slots whose state differs after k
    cause: list = field(default_factory=list)       # explanations found
    note: str = ""


def _ancestors(q: np.ndarray, seed: int, lane: int, m: int) -> np.ndarray:
    w = pf_oracle.philox4x32_10([0, 0xFFFFFFFF, lane, m], [seed & 0xFFFFFFFF, seed >> 32])
    r64 = (int(w[1]) << 32) | int(w[0])
    return pf_oracle.resample_systematic(q, r64)


def fragile_weights(e_prev: np.ndarray, svar: bool) -> list[tuple[int, int]]:
    """(particle, direction) of integer weights that a last-place difference
    of exp could move by one: frac(2^32 exp(e - max e)) within 2^-20 of 0
    (direction -1) or of 1 (+1)."""
    e = np.asarray(e_prev, np.float64)
    if svar:
        e = pf_oracle.grid20(e)
    emax = float(e.max())
    out = []
    for i, ei in enumerate(e):
        v = math.ldexp(math.exp(float(ei) - emax), 32)
        f = v - math.floor(v)
        if f < 2.0 ** -20 and v >= 1.0:
            out.append((i, -1))
        elif f > 1.0 - 2.0 ** -20:
            out.append((i, +1))
    return out


def trace_filter(pf, net, theta, m: int, t: int, x0, obs_times, y, C, sigma, N: int, seed: int,
                 model=None, cluster_blocks: int = 0, budget: int = pf_oracle.DEFAULT_BUDGET,
                 gpu_run=None) -> Report:
    """Trace the filter (theta row `theta` with id m, trajectory t of y
    [T][K][P]).  gpu_run(Kp) -> dict(status, events, digest, final_states
    [N][U]) overrides the GPU side (used to test the harness on the CPU)."""
    theta = np.asarray(theta, np.float64).reshape(-1)
    obs_times = np.asarray(obs_times, np.float64)
    y = np.asarray(y, np.float64)
    K = len(obs_times)
    svar = bool(model and model.get("obs_var") is not None)
    rate_coef = None if not model else model.get("rate_coef")

    if gpu_run is None:
        def gpu_run(Kp):
            g = pf.pf_loglik(net, theta[None, :], x0, obs_times[:Kp], y[:, :Kp], C, sigma, N,
                             seed, diagnostics=True, final_states=True,
                             theta_ids=np.array([m]), model=model, event_budget=budget,
                             cluster_blocks=cluster_blocks)
            return {"status": int(g["status"][0]), "events": int(g["events"][0, t]),
                    "digest": int(g["digest"][0, t]), "final_states": g["final_states"][0, t]}

    def oracle_run(Kp):
        o = pf_oracle.pf_loglik(net, theta[None, :], x0, obs_times[:Kp], y[t:t + 1, :Kp], C, sigma,
                                N, seed, theta_ids=[m], traj_ids=[t], want_final_states=True,
                                model=model, budget=budget)
        return {"status": int(o["status"][0]), "events": int(o["events"][0, 0]),
                "digest": int(o["digest"][0, 0]), "final_states": o["final_states"][0, 0]}

    def same(a, b):
        return (a["status"] == b["status"] and a["events"] == b["events"]
                and a["digest"] == b["digest"])

    full_g, full_o = gpu_run(K), oracle_run(K)
    if same(full_g, full_o):
        return Report(False, note="histories agree; the difference is in the log-likelihood only")
    lo, hi = 0, K            # prefix lo agrees (0: trivially), prefix hi disagrees
    while hi - lo > 1:
        mid = (lo + hi) // 2
        if same(gpu_run(mid), oracle_run(mid)):
            lo = mid
        else:
            hi = mid
    k = hi - 1
    g = gpu_run(hi)
    tr = pf_oracle.pf_trace(net, theta, m, t, x0, obs_times[:hi], y[t, :hi], C, sigma, N, seed,
                            k_trace=k, budget=budget, model=model)
    G = np.asarray(g["final_states"], np.int64)
    bad = np.flatnonzero((G != tr["x_end"]).any(axis=1)).tolist()
    rep = Report(False, k=k, particles=bad)
    if g["status"] != 0 or tr["status"] != 0:
        rep.note = f"status differs at interval {k}: GPU {g['status']}, oracle {tr['status']}"
        return rep
    lane = (t << 20) | k
    t0 = float(obs_times[k - 1]) if k > 0 else 0.0
    t1 = float(obs_times[k])

    def replay(x, i, alt_draw=-1, alt_kind=0):
        return pf_oracle.ssa_replay(net, theta, x, t0, t1, seed, i, lane, m, budget=budget,
                                    alt_draw=alt_draw, alt_kind=alt_kind, rate_coef=rate_coef)

    # (a) an integer weight of interval k-1 off by one
    if k > 0:
        before = pf_oracle.pf_trace(net, theta, m, t, x0, obs_times[:k], y[t, :k], C, sigma, N,
                                    seed, k_trace=k - 1, budget=budget, model=model)["x_end"]
        for i, step in fragile_weights(tr["e_prev"], svar):
            q = tr["q_prev"].copy()
            q[i] = np.uint64(int(q[i]) + step)
            anc = _ancestors(q, seed, lane, m)
            if np.array_equal(anc, tr["anc"]):
                continue
            ends = np.array([replay(before[anc[j]], j)[0] for j in range(N)])
            if np.array_equal(ends, G):
                rep.cause.append(("integer weight", k - 1, i, step))
                rep.traced = True
                return rep
    # (b) one draw of a mismatching particle
    explained = []
    for i in bad:
        xe, _, _, rec = replay(tr["x_start"][i], i)
        assert np.array_equal(xe, tr["x_end"][i])
        found = None
        for r in rec:
            j, flags = int(r[0]), int(r[6])
            alts = []
            if flags & RP_WEDGE and r[7] <= FRAGILE_ULPS:
                alts.append(ALT_WEDGE_FLIP)
            if flags & RP_TAIL:
                alts += [ALT_E_UP, ALT_E_DOWN]
            if r[8] <= FRAGILE_ULPS:
                alts.append(ALT_TIME_FLIP)
            if r[9] <= FRAGILE_ULPS:
                alts += [ALT_CHOSEN_UP, ALT_CHOSEN_DOWN]
            for alt in alts:
                xa = replay(tr["x_start"][i], i, alt_draw=j, alt_kind=alt)[0]
                if np.array_equal(xa, G[i]):
                    found = ("draw", k, i, j, alt)
                    break
            if found:
                break
        if found is None:
            rep.note = f"particle {i} of interval {k} is not explained by a last-place difference"
            return rep
        explained.append(found)
    rep.cause = explained
    rep.traced = bool(bad)
    if not bad:
        rep.note = "states agree but the history digest differs (ancestors)"
    return rep
