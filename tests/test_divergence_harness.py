"""The first-divergence harness (tests/divergence.py) on the CPU.

Its GPU side is replaced by copies of the oracle with a planted difference,
so that the divergence is known: a time test that fires an event lying exactly
on the observation time (a last-place tie the harness must find and explain
as such) and a state changed outright (a real bug it must refuse to
explain).  Its oracle replay is pinned to the oracle's own filter."""
from __future__ import annotations

import math

import numpy as np
import pytest

from oracle import pf_oracle
from paper_1606_08281_gb300 import workloads as W
from tests import divergence as D


def variant_run(variant, w, theta, m, t, obs_times, y, N, seed):
    def run(Kp):
        o = variant.pf_loglik(w.net, theta[None, :], w.x0, obs_times[:Kp], y[t:t + 1, :Kp], w.C,
                              w.sigma, N, seed, theta_ids=[m], traj_ids=[t],
                              want_final_states=True, model=w.model)
        return {"status": int(o["status"][0]), "events": int(o["events"][0, 0]),
                "digest": int(o["digest"][0, 0]), "final_states": o["final_states"][0, 0]}
    return run


@pytest.mark.parametrize("name,k", [("gene_expression", 3), ("cascade", 2), ("lac_gfp", 1)])
def test_replay_reproduces_the_oracle_interval(name, k):
    """Every particle of an interval, replayed draw by draw from its start
    state, ends in the oracle's state with the oracle's event count."""
    w = W.get(name).subset(T=2, K=k + 1)
    th = w.thetas(3)[2]
    N = 40
    tr = pf_oracle.pf_trace(w.net, th, 2, 1, w.x0, w.obs_times, w.observations()[1], w.C, w.sigma,
                            N, 5, k_trace=k, model=w.model)
    o = pf_oracle.pf_loglik(w.net, th[None], w.x0, w.obs_times, w.observations()[1:2], w.C,
                            w.sigma, N, 5, theta_ids=[2], traj_ids=[1], want_final_states=True,
                            model=w.model)
    assert tr["digest"] == o["digest"][0, 0] and tr["events"] == o["events"][0, 0]
    assert np.array_equal(tr["x_end"], o["final_states"][0, 0])
    t0 = w.obs_times[k - 1] if k else 0.0
    rc = None if not w.model else w.model.get("rate_coef")
    for i in range(N):
        xe, fired, st, _ = pf_oracle.ssa_replay(w.net, th, tr["x_start"][i], t0, w.obs_times[k], 5,
                                                i, (1 << 20) | k, 2, rate_coef=rc)
        assert st == 0 and fired == tr["fired"][i]
        assert np.array_equal(xe, tr["x_end"][i]), i
    if k:
        assert np.array_equal(D._ancestors(tr["q_prev"], 5, (1 << 20) | k, 2), tr["anc"])


def test_harness_finds_and_explains_a_time_tie(tmp_path):
    """Put observation time k exactly on an event time of particle i; a copy of
    the oracle whose time test also stops on equality then leaves the oracle
    at (k, i, that draw), and the harness explains it as the time test's
    last-place tie."""
    w = W.gene_expression().subset(T=2, K=6)
    th, m, t, N, seed, k, i = w.thetas(2)[1], 1, 1, 30, 8, 3, 7
    y = w.observations()
    tr = pf_oracle.pf_trace(w.net, th, m, t, w.x0, w.obs_times, y[t], w.C, w.sigma, N, seed,
                            k_trace=k)
    _, _, _, rec = pf_oracle.ssa_replay(w.net, th, tr["x_start"][i], w.obs_times[k - 1],
                                        w.obs_times[k], seed, i, (t << 20) | k, m)
    fired = rec[rec[:, 5] >= 0]
    assert len(fired) >= 3
    j = int(fired[len(fired) // 2, 0])
    times = w.obs_times.copy()
    times[k] = fired[len(fired) // 2, 4]                 # an event exactly at t_k
    src = pf_oracle.source_text()
    old = "if (t_next > t_end) return ORC_OK;"
    assert src.count(old) == 1
    variant = pf_oracle.compile_variant(src.replace(old, "if (t_next >= t_end) return ORC_OK;"),
                                        tmp_path)
    rep = D.trace_filter(None, w.net, th, m, t, w.x0, times, y, w.C, w.sigma, N, seed,
                         gpu_run=variant_run(variant, w, th, m, t, times, y, N, seed))
    assert rep.traced, rep
    assert rep.k == k and rep.particles == [i]
    assert rep.cause == [("draw", k, i, j, D.ALT_TIME_FLIP)]


def test_harness_refuses_to_explain_a_real_difference(tmp_path):
    """A copy of the oracle that adds one molecule to particle 3 after
    interval 2: the harness locates it and reports it as unexplained."""
    w = W.gene_expression().subset(T=2, K=6)
    th, m, t, N, seed = w.thetas(2)[0], 0, 0, 30, 9
    src = pf_oracle.source_text()
    old = "        for (int j = 0; j < N; j++)\n            digest += slot_digest("
    assert src.count(old) == 1
    planted = "        if (k == 2) x[3 * (size_t)U] += 1;\n" + old
    variant = pf_oracle.compile_variant(src.replace(old, planted), tmp_path)
    rep = D.trace_filter(None, w.net, th, m, t, w.x0, w.obs_times, w.observations(), w.C, w.sigma,
                         N, seed, gpu_run=variant_run(variant, w, th, m, t, w.obs_times,
                                                      w.observations(), N, seed))
    assert not rep.traced
    assert rep.k == 2 and rep.particles == [3]


def test_fragile_weights_are_those_within_two_ulps_of_an_integer():
    """2^32 exp(log 0.5) is 2^31 or one unit below it (fragile); 2^32 / e has a
    fractional part near 0.7 (not fragile)."""
    e = np.array([0.0, math.log(0.5), -1.0])
    got = dict(D.fragile_weights(e, svar=False))
    assert 1 in got and 2 not in got
    v = math.ldexp(math.exp(e[1]), 32)
    assert got[1] == (-1 if v == 2.0 ** 31 else +1)
