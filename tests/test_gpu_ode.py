"""The CUDA ODE likelihood of the Egf-Ras-Raf-Mek-Erk model (pf_erk_loglik,
through the C ABI) against the ODE oracle (oracle/ode.py, scipy DOP853).

Tolerance, derived from the solvers' settings: the kernel runs at
rtol 1e-12 / atol 1e-15 here and the oracle at rtol 1e-11 / atol 1e-14, so
the states agree to ~1e-10 relative; allowing 100x for the accumulation over
the trajectory, the FRET ratio R (a quotient of two such states) agrees to
eps_R = 2e-8 relative, and each log-density term log N(y; R, sigma^2) to
|y - R| eps_R |R| / sigma^2 + (eps_R |R| / sigma)^2.  The per-pattern values
must agree within the sum of those terms over the observation times (plus
1e-12 relative).
"""
from __future__ import annotations

import numpy as np
import pytest

from oracle import ode
from paper_1606_08281_gb300 import workloads as W

pytestmark = pytest.mark.gpu
EPS_R = 2e-8


@pytest.fixture(scope="module")
def pf():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1606_08281_gb300 import build, pf as pfmod
    build.build()
    pfmod.load()
    return pfmod


def tolerance(th, R, y):
    s = th[32]
    return (np.abs(y - R) * EPS_R * np.abs(R) / s ** 2 + (EPS_R * np.abs(R) / s) ** 2).sum()


def check_rows(g, thetas, w, y):
    assert (g["status"] == 0).all(), g["status"]
    for m, th in enumerate(thetas):
        Rm = ode.observe(th, w.patterns, w.obs_times)
        _, per = ode.loglik(th, w.patterns, w.obs_times, y)
        for p in range(len(w.patterns)):
            tol = tolerance(th, Rm[p], y[p]) + 1e-12 * abs(per[p])
            assert abs(g["ll_pattern"][m, p] - per[p]) <= tol, (m, p, g["ll_pattern"][m, p], per[p], tol)
        assert abs(g["loglik"][m] - per.sum()) <= sum(
            tolerance(th, Rm[p], y[p]) for p in range(len(w.patterns))) + 1e-12 * abs(per.sum())


def test_theta_bar_and_neighbourhood(pf):
    w = W.erk()
    th = np.vstack([w.theta_bar, w.thetas(11)])
    y = w.observations()
    g = pf.pf_erk_loglik(th, w.patterns, w.obs_times, y, rtol=1e-12, atol=1e-15, diagnostics=True)
    check_rows(g, th, w, y)
    assert (g["steps"] > 0).all()


def test_noise_free_data_score_the_normaliser(pf):
    w = W.erk()
    th = w.theta_bar
    y = ode.observe(th, w.patterns, w.obs_times)
    g = pf.pf_erk_loglik(th[None, :], w.patterns, w.obs_times, y, rtol=1e-12, atol=1e-15)
    want = -y.size * (np.log(th[32]) + 0.5 * np.log(2 * np.pi))
    assert abs(g["loglik"][0] - want) < sum(tolerance(th, y[p], y[p]) for p in range(len(y))) + 1e-9


def test_default_tolerance_close(pf):
    """At the default rtol 1e-10 the values stay within 100x the bound."""
    w = W.erk()
    th = w.thetas(4)
    y = w.observations()
    g = pf.pf_erk_loglik(th, w.patterns, w.obs_times, y, diagnostics=True)
    for m in range(len(th)):
        _, per = ode.loglik(th[m], w.patterns, w.obs_times, y)
        Rm = ode.observe(th[m], w.patterns, w.obs_times)
        tol = 100 * sum(tolerance(th[m], Rm[p], y[p]) for p in range(len(y))) + 1e-9 * abs(per.sum())
        assert abs(g["loglik"][m] - per.sum()) <= tol


def test_invalid_rows_budget_and_device_mode(pf):
    import torch
    w = W.erk()
    th = np.vstack([w.theta_bar] * 3)
    th[1, 5] = -1.0                      # a negative constant
    th[2, 33] = 1.2                      # FRET efficiency >= 1
    y = w.observations()
    r = pf.pf_erk_loglik(th, w.patterns, w.obs_times, y)
    assert r["status"].tolist() == [0, pf.PF_ST_INVALID_THETA, pf.PF_ST_INVALID_THETA]
    b = pf.pf_erk_loglik(th[:1], w.patterns, w.obs_times, y, max_steps=20)
    assert b["status"][0] == pf.PF_ST_BUDGET and np.isneginf(b["loglik"][0])
    dev = torch.device("cuda:0")
    d = pf.pf_erk_loglik(torch.from_numpy(th).to(dev), w.patterns, w.obs_times,
                         torch.from_numpy(y).to(dev))
    torch.cuda.synchronize()
    assert np.array_equal(d["loglik"].cpu().numpy()[:1], r["loglik"][:1])
    with pytest.raises(pf.PfError):
        pf.pf_erk_loglik(th, w.patterns, np.array([0.0, 1.0]), y[:, :2])   # obs_times[0] = 0


def test_prior_draws_finish(pf):
    """Draws from the whole prior (rates over 15 e-folds): every row ends OK
    or BUDGET (stiff for an explicit method), finite when OK."""
    w = W.erk()
    th = w.prior_thetas(256)
    g = pf.pf_erk_loglik(th, w.patterns, w.obs_times, w.observations(), max_steps=20000)
    assert set(np.unique(g["status"]).tolist()) <= {0, pf.PF_ST_BUDGET}
    assert np.isfinite(g["loglik"][g["status"] == 0]).all()


def test_full_size_erk_sampled(pf):
    """The bench's launch: all 4096 theta rows x 6 patterns at the default
    tolerance; 6 sampled rows against the oracle within 100x the bound."""
    w = W.erk()
    th = w.thetas()
    y = w.observations()
    g = pf.pf_erk_loglik(th, w.patterns, w.obs_times, y)
    assert (g["status"] == 0).all()
    for m in np.random.default_rng(6).choice(len(th), 6, replace=False):
        _, per = ode.loglik(th[m], w.patterns, w.obs_times, y)
        Rm = ode.observe(th[m], w.patterns, w.obs_times)
        tol = 100 * sum(tolerance(th[m], Rm[p], y[p]) for p in range(len(y))) + 1e-9 * abs(per.sum())
        assert abs(g["loglik"][m] - per.sum()) <= tol, (m, g["loglik"][m], per.sum(), tol)
    # 4096 rows need more lane pairs than one wave holds and run on persistent
    # pairs, 64 rows on one pair each: the same rows give the same bits
    sub = pf.pf_erk_loglik(th[:64], w.patterns, w.obs_times, y)
    assert np.array_equal(sub["loglik"], g["loglik"][:64])


def test_persistent_pairs_equal_one_wave(pf):
    """More problems than one resident wave (4096 and 16 384 rows x 6
    patterns) run on persistent lane pairs fed by a work counter, the block
    moving its busy problems onto its lowest pairs once the counter is
    exhausted; each problem's result is the one the one-wave kernel gives for
    the same row (3000 rows: 18 000 problems, one pair each), bit for bit."""
    w = W.erk()
    w.M = 16384
    th = w.thetas()
    y = w.observations()
    small = pf.pf_erk_loglik(th[:3000], w.patterns, w.obs_times, y, diagnostics=True)
    assert (small["status"] == 0).all()
    for M in (4096, 16384):
        big = pf.pf_erk_loglik(th[:M], w.patterns, w.obs_times, y, diagnostics=True)
        assert (big["status"] == 0).all()
        assert np.array_equal(big["loglik"][:3000], small["loglik"]), M
        assert np.array_equal(big["steps"][:3000], small["steps"]), M
