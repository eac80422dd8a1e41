"""The CUDA FSP likelihood (pf_fsp_loglik, through the C ABI) against the FSP
oracle (oracle/fsp.py, scipy's sparse matrix-exponential action).

Tolerance: the kernel truncates each uniformization series where the Poisson
tail is below 1e-17 and sums at most ~2000 terms of size <= 1 per sub-step in
FP64 (rounding ~2000 * 2^-53 ~ 2e-13 of a factor), over at most 50
observation times; scipy's expm_multiply is accurate to about 1e-15.  So the
per-trajectory log-likelihoods must agree to 1e-9 relative, the dropped mass
(leak) to 1e-9 absolute.
"""
from __future__ import annotations

import numpy as np
import pytest

from oracle import fsp
from paper_1606_08281_gb300 import workloads as W

pytestmark = pytest.mark.gpu

RTOL = 1e-9
DIMER = {"reactants": np.array([[0], [2]], np.int32), "products": np.array([[1], [0]], np.int32),
         "rate_index": None}


@pytest.fixture(scope="module")
def pf():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1606_08281_gb300 import build, pf as pfmod
    build.build()
    pfmod.load()
    return pfmod


def both(pf, net, th, x0, box, times, y, C, sigma, model=None):
    g = pf.pf_fsp_loglik(net, th, x0, box, times, y, C, sigma, model=model, diagnostics=True)
    tot, ll, leak = fsp.loglik_batch(net, th, x0, box, times, y, C, sigma, model)
    assert (g["status"] == 0).all(), g["status"]
    np.testing.assert_allclose(g["ll_traj"], ll, rtol=RTOL, atol=0)
    np.testing.assert_allclose(g["loglik"], tot, rtol=RTOL, atol=0)
    np.testing.assert_allclose(g["leak"], leak, rtol=0, atol=1e-9)
    return g


def test_birth_death_prior_draws(pf):
    """12 theta rows of the birth-death batch on the box 0..1200 (stationary
    means up to several hundred, lambda dt up to ~1000)."""
    w = W.birth_death()
    th = w.thetas(12)
    both(pf, w.net, th, w.x0, w.fsp_box, w.obs_times, w.observations(), w.C, w.sigma)


def test_telegraph_prior_draws(pf):
    w = W.telegraph()
    th = w.thetas(64)
    both(pf, w.net, th, w.x0, w.fsp_box, w.obs_times, w.observations(), w.C, w.sigma)


def test_gene_expression_small_box(pf):
    """Two species (8 x 120 states), two trajectories, mass leaving the box."""
    w = W.gene_expression()
    th = np.array([[0.1, 0.1, 1.0, 0.01], [0.3, 0.2, 2.0, 0.05], [0.05, 0.5, 5.0, 0.1]])
    g = both(pf, w.net, th, w.x0, [7, 119], w.obs_times[:10], w.observations()[:2, :10], w.C,
             w.sigma)
    assert g["leak"].max() > 0.0


def test_second_order_network(pf):
    rng = np.random.default_rng(3)
    times = np.array([0.5, 1.0, 2.5, 4.0])
    y = rng.normal(size=(2, 4, 1)) * 2.0 + 12.0
    both(pf, DIMER, [[3.0, 0.05], [1.0, 0.2]], [20], [60], times, y, [[1.0]], [1.5])


def test_model_extensions(pf):
    """Composed rate, uniform initial counts, offset and state-dependent variance."""
    w = W.birth_death()
    model = {"rate_coef": [[1.0, 3.0, 0.0], [0.0, 0.0, 1.0]], "x0_hi": [15], "obs_offset": [2.0],
             "obs_var": [[0.5]]}
    th = W.log_uniform(np.random.default_rng(12), [1.0, 0.1, 0.05], [20.0, 5.0, 1.0], 9)
    y = w.observations() * 1.5 + 2.0
    both(pf, w.net, th, [5], [400], w.obs_times, y, [[1.5]], [1.0], model)


def test_observation_at_time_zero(pf):
    y = np.array([[[3.3], [2.0]]])
    both(pf, W.birth_death_network(), [[10.0, 0.2]], [2], [100], [0.0, 1.0], y, [[1.0]], [1.7])


def test_device_pointers_match_host(pf):
    import torch
    w = W.telegraph()
    th = w.thetas(32)
    h = pf.pf_fsp_loglik(w.net, th, w.x0, w.fsp_box, w.obs_times, w.observations(), w.C, w.sigma)
    dev = torch.device("cuda:0")
    g = pf.pf_fsp_loglik(w.net, torch.from_numpy(th).to(dev), w.x0, w.fsp_box, w.obs_times,
                         torch.from_numpy(w.observations()).to(dev), w.C, w.sigma)
    torch.cuda.synchronize()
    assert np.array_equal(g["loglik"].cpu().numpy(), h["loglik"])


def test_invalid_rows_and_arguments(pf):
    w = W.telegraph()
    th = w.thetas(3)
    th[1, 0] = -1.0
    r = pf.pf_fsp_loglik(w.net, th, w.x0, w.fsp_box, w.obs_times, w.observations(), w.C, w.sigma)
    assert r["status"].tolist() == [0, pf.PF_ST_INVALID_THETA, 0]
    assert np.isnan(r["loglik"][1]) and np.isfinite(r["loglik"][[0, 2]]).all()
    with pytest.raises(pf.PfError):   # x0 outside the box
        pf.pf_fsp_loglik(w.net, th, [0, 1, 70], w.fsp_box, w.obs_times, w.observations(), w.C,
                         w.sigma)
    with pytest.raises(pf.PfError):   # too many states
        pf.pf_fsp_loglik(w.net, th, w.x0, [1, 1, 5000], w.obs_times, w.observations(), w.C,
                         w.sigma)
    e = pf.pf_fsp_loglik(w.net, np.zeros((0, 4)), w.x0, w.fsp_box, w.obs_times, w.observations(),
                         w.C, w.sigma)
    assert e["loglik"].shape == (0,)


def test_gpu_filter_unbiased_for_gpu_fsp(pf):
    """The CUDA particle filter is unbiased for exp of the CUDA FSP value: 400
    rows of theta* (independent random streams) on the telegraph workload."""
    w = W.telegraph()
    L = pf.pf_fsp_loglik(w.net, w.theta_star[None, :], w.x0, w.fsp_box, w.obs_times,
                         w.observations(), w.C, w.sigma)["loglik"][0]
    th = np.repeat(w.theta_star[None, :], 400, axis=0)
    r = pf.pf_loglik(w.net, th, w.x0, w.obs_times, w.observations(), w.C, w.sigma, 200, 77)
    z = np.exp(r["loglik"] - L)
    se = z.std(ddof=1) / np.sqrt(len(z))
    assert abs(z.mean() - 1.0) < 4 * se + 1e-3, (z.mean(), se)


def test_full_size_telegraph_sampled(pf):
    """The bench's launch: all 4096 theta rows of the telegraph workload at
    once; 16 sampled rows against the oracle."""
    w = W.telegraph()
    th = w.thetas()
    g = pf.pf_fsp_loglik(w.net, th, w.x0, w.fsp_box, w.obs_times, w.observations(), w.C, w.sigma)
    assert (g["status"] == 0).all()
    pick = np.random.default_rng(5).choice(len(th), 16, replace=False)
    tot, _, _ = fsp.loglik_batch(w.net, th[pick], w.x0, w.fsp_box, w.obs_times, w.observations(),
                                 w.C, w.sigma)
    np.testing.assert_allclose(g["loglik"][pick], tot, rtol=RTOL, atol=0)
