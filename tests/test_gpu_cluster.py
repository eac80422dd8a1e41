"""Filters split over a thread-block cluster (pf_options.cluster_blocks = C,
2..8 blocks on as many SMs) against the oracle and the one-block filter.

Same bar as test_gpu_parity: per filter the fired reactions, the history
digest, the statuses and the final states are bit-identical to the oracle's
(the integer weights, their prefix sums and the ancestors are exact integer
work, however the population is split); log-likelihoods agree within 1e-9
relative.  Against the one-block filter the log-likelihoods differ only by
the summation order of the weights: within 1e-12 relative.
"""
from __future__ import annotations

import numpy as np
import pytest

from oracle import pf_oracle
from paper_1606_08281_gb300 import workloads as W

pytestmark = pytest.mark.gpu

RTOL = 1e-9


@pytest.fixture(scope="module")
def pf():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1606_08281_gb300 import build, pf as pfmod
    build.build()
    pfmod.load()
    return pfmod


def check(pf, w_net, th, x0, times, y, C, sigma, N, seed, cb, model=None, budget=0,
          final_states=True, block_threads=0):
    g = pf.pf_loglik(w_net, th, x0, times, y, C, sigma, N, seed, diagnostics=True,
                     final_states=final_states, cluster_blocks=cb, model=model,
                     event_budget=budget, block_threads=block_threads)
    o = pf_oracle.pf_loglik(w_net, th, x0, times, y, C, sigma, N, seed, model=model,
                            budget=budget or pf_oracle.DEFAULT_BUDGET,
                            want_final_states=final_states)
    assert (g["status"] == o["status"]).all(), (g["status"], o["status"])
    ok = o["status"] == 0
    bad = np.argwhere(~((g["events"] == o["events"]) & (g["digest"] == o["digest"]))[ok])
    assert len(bad) == 0, f"history mismatch in filters {bad[:10].tolist()}"
    np.testing.assert_allclose(g["ll_traj"][ok], o["ll_traj"][ok], rtol=RTOL, atol=0)
    np.testing.assert_allclose(g["loglik"][ok], o["loglik"][ok], rtol=RTOL, atol=0)
    assert np.isneginf(g["loglik"][o["status"] == 1]).all()
    if final_states:
        assert (g["final_states"][ok] == o["final_states"][ok]).all()
    one = pf.pf_loglik(w_net, th, x0, times, y, C, sigma, N, seed, diagnostics=True, model=model,
                       event_budget=budget)
    assert (one["status"] == g["status"]).all()
    assert (one["digest"][ok] == g["digest"][ok]).all() and (one["events"][ok] == g["events"][ok]).all()
    np.testing.assert_allclose(one["ll_traj"][ok], g["ll_traj"][ok], rtol=1e-12, atol=0)
    return g


@pytest.mark.parametrize("cb,N", [(2, 1000), (3, 1000), (4, 257), (8, 1000), (8, 37), (5, 6),
                                  (8, 16384)])
def test_gene_expression_split(pf, cb, N):
    """Even and ragged shares (N = 37 over 8 blocks: 5 particles each, 2 in
    the last block; N = 6 over 5 blocks: 2, 2, 2, 0 -> rejected, see below),
    and the maximum population (16384 particles, 2048 per block; the one-block
    filter it is compared with runs from the global-memory slab)."""
    w = W.gene_expression().subset(T=2, K=8)
    if N - (cb - 1) * -(-N // cb) < 1:
        with pytest.raises(pf.PfError) as e:
            pf.pf_loglik(w.net, w.thetas(2), w.x0, w.obs_times, w.observations(), w.C, w.sigma,
                         N, 7, cluster_blocks=cb)
        assert e.value.code == pf.PF_EINVAL
        return
    check(pf, w.net, w.thetas(6), w.x0, w.obs_times, w.observations(), w.C, w.sigma, N, 7, cb)


def test_cascade_split(pf):
    """10 species / 20 reactions (states in shared memory, dependency lists)."""
    w = W.cascade().subset(T=2, K=5)
    check(pf, w.net, w.thetas(4), w.x0, w.obs_times, w.observations(), w.C, w.sigma, 512, 13, 4)


def test_lac_gfp_split(pf):
    """Model extensions: uniform random initial counts (keyed by the particle's
    index in the filter), composed rates, state-dependent variance."""
    w = W.lac_gfp()
    th = np.vstack([w.theta_star, w.thetas(3)])
    check(pf, w.net, th, w.x0, w.obs_times[:4], w.observations()[:2, :4], w.C, w.sigma, 200,
          w.filter_seed, 4, model=w.model)


def test_small_blocks_and_observation_at_zero(pf):
    w = W.birth_death()
    y = np.array([[[3.3], [7.0], [6.1]]])
    check(pf, w.net, w.thetas(5), w.x0, [0.0, 0.25, 1.5], y, w.C, w.sigma, 100, 3, 2,
          block_threads=32)


def test_budget_and_invalid_rows(pf):
    w = W.birth_death()
    th = w.thetas(8).copy()
    check(pf, w.net, th, w.x0, w.obs_times, w.observations(), w.C, w.sigma, 64, 5, 4, budget=30)
    th[1, 0] = -1.0
    g = pf.pf_loglik(w.net, th, w.x0, w.obs_times, w.observations(), w.C, w.sigma, 64, 5,
                     cluster_blocks=4)
    assert g["status"][1] == pf.PF_ST_INVALID_THETA and np.isnan(g["loglik"][1])


def test_early_rejection_split(pf):
    """The level-set threshold with split filters: rows below it REJECTED,
    the others exactly the split filter's full values."""
    w = W.gene_expression().subset(T=3, K=12)
    th = w.thetas(32)
    full = pf.pf_loglik(w.net, th, w.x0, w.obs_times, w.observations(), w.C, w.sigma, 300, 31,
                        diagnostics=True, cluster_blocks=3)
    thr = float(np.median(full["loglik"]))
    cut = pf.pf_loglik(w.net, th, w.x0, w.obs_times, w.observations(), w.C, w.sigma, 300, 31,
                       diagnostics=True, reject_below=thr, cluster_blocks=3)
    below = full["loglik"] < thr
    assert (cut["status"][below] == pf.PF_ST_REJECTED).all()
    assert (cut["status"][~below] == 0).all()
    assert np.array_equal(cut["loglik"][~below], full["loglik"][~below])
    assert cut["events"].sum() < full["events"].sum()


def test_bad_cluster_sizes(pf):
    w = W.birth_death()
    for cb in (-1, 9):
        with pytest.raises(pf.PfError) as e:
            pf.pf_loglik(w.net, w.thetas(2), w.x0, w.obs_times, w.observations(), w.C, w.sigma,
                         64, 5, cluster_blocks=cb)
        assert e.value.code == pf.PF_EINVAL
    # a share too large for shared memory (16384 cascade particles over 2 blocks)
    c = W.cascade().subset(T=1, K=2)
    with pytest.raises(pf.PfError) as e:
        pf.pf_loglik(c.net, c.thetas(1), c.x0, c.obs_times, c.observations(), c.C, c.sigma,
                     16384, 5, cluster_blocks=2)
    assert e.value.code == pf.PF_EINVAL
