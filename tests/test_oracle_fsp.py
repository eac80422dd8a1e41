"""Pins of the FSP oracle (oracle/fsp.py): the exact (truncated) likelihood
by the finite state projection, which the CUDA FSP kernel is compared with.

Each pin ties it to something other than itself: the closed-form
birth-death transition law (a second route, oracle/exact_bd.py), the moment
equations of the RNA telegraph model, conservation laws, the empirical law of
the SSA oracle on a second-order network, and the particle-filter oracle's
unbiasedness for exp(log-likelihood).  Planted mistakes in a copy of fsp.py
must each fail a pin.
"""
from __future__ import annotations

import types

import numpy as np
import pytest
from scipy import stats

from oracle import exact_bd, fsp, pf_oracle
from paper_1606_08281_gb300 import workloads as W

BD = W.birth_death_network()
TG = W.telegraph_network()
DIMER = {"reactants": np.array([[0], [2]], np.int32), "products": np.array([[1], [0]], np.int32),
         "rate_index": None}     # 0 -> X (c1), X + X -> 0 (c2 x(x-1)/2)


def check_birth_death_closed_form(f):
    """FSP on 0..200 equals the forward algorithm with the closed-form
    Binomial (+) Poisson transition, with and without the model extensions."""
    w = W.birth_death()
    y = w.observations()[0, :, 0] * 1.3 + 0.5
    for k1, k2 in [(10.0, 0.2), (14.0, 0.3), (5.0, 0.1)]:
        want, _ = exact_bd.loglik(k1, k2, 10, w.obs_times, y, c=1.3, sigma=1.5, nmax=200,
                                  transition=exact_bd.transition_closed)
        got, leak = f.loglik(BD, [k1, k2], [10], [200], w.obs_times, y[:, None], [[1.3]], [1.5])
        assert abs(leak) < 1e-12
        assert np.isclose(got, want, rtol=1e-10, atol=0), (k1, k2, got, want)
    model = {"x0_hi": [15], "obs_offset": [2.0], "obs_var": [[0.5]]}
    want, _ = exact_bd.loglik(10.0, 0.2, 5, w.obs_times, y, c=1.3, sigma=1.5, nmax=200,
                              transition=exact_bd.transition_closed, x0_hi=15, obs_offset=2.0,
                              obs_var=0.5)
    got, _ = f.loglik(BD, [10.0, 0.2], [5], [200], w.obs_times, y[:, None], [[1.3]], [1.5], model)
    assert np.isclose(got, want, rtol=1e-10, atol=0)


def test_birth_death_equals_closed_form_route():
    check_birth_death_closed_form(fsp)


def telegraph_means(th, t):
    """Moment equations of the telegraph model from G_off = 1, RNA = 0:
    g' = th1 (1 - g) - th2 g,  m' = th3 g - th4 m."""
    s = th[0] + th[1]
    ginf = th[0] / s
    g = ginf * (1.0 - np.exp(-s * t))
    m = (th[2] * ginf / th[3] * (1.0 - np.exp(-th[3] * t))
         - th[2] * ginf * (np.exp(-s * t) - np.exp(-th[3] * t)) / (th[3] - s))
    return g, m


def check_telegraph_moments(f):
    """Means of the propagated distribution follow the moment equations;
    G_on + G_off = 1 on the support; no mass leaves a large enough box."""
    th = np.array([0.05, 0.1, 2.0, 0.1])
    box = [1, 1, 90]
    X = f.box_states(box)
    Q = f.generator(TG, th, box)
    for t in [3.0, 20.0, 80.0]:
        a = f.propagate(Q, f.initial([0, 1, 0], box), t)
        assert abs(a.sum() - 1.0) < 1e-12
        assert a[X[:, 0] + X[:, 1] != 1].max(initial=0.0) < 1e-300
        g, m = telegraph_means(th, t)
        assert np.isclose(a @ X[:, 0], g, rtol=1e-9), (t, a @ X[:, 0], g)
        assert np.isclose(a @ X[:, 2], m, rtol=1e-9), (t, a @ X[:, 2], m)


def test_telegraph_moment_equations():
    check_telegraph_moments(fsp)


def check_second_order_law(f, n=20000):
    """X + X -> 0 with propensity c2 x(x-1)/2: the FSP law at t matches the
    empirical law of the SSA oracle's paths (chi-square)."""
    th = [3.0, 0.05]
    box = [60]
    t = 2.5
    a = f.propagate(f.generator(DIMER, th, box), f.initial([20], box), t)
    states, _, _ = pf_oracle.ssa_paths(DIMER, th, [20], [t], n, seed=99)
    cnt = np.bincount(states[:, 0, 0], minlength=61)[:61]
    exp = a * n
    keep = exp > 5
    chi = ((cnt[keep] - exp[keep]) ** 2 / exp[keep]).sum()
    assert stats.chi2.sf(chi, keep.sum() - 1) > 1e-4, chi


def test_second_order_law_matches_ssa():
    check_second_order_law(fsp)


def check_filter_unbiased(f, S=300):
    """The particle filter is unbiased for the likelihood: over seeds,
    mean exp(ll_PF - L_FSP) = 1 on the telegraph workload."""
    w = W.telegraph()
    y = w.observations()
    for th in [w.theta_star, np.array([0.003, 0.002, 0.06, 0.002])]:
        L, leak = f.loglik(w.net, th, w.x0, w.fsp_box, w.obs_times, y[0], w.C, w.sigma)
        assert abs(leak) < 1e-12
        lls = np.array([pf_oracle.pf_loglik(w.net, [th], w.x0, w.obs_times, y, w.C, w.sigma, 200,
                                            500 + s)["loglik"][0] for s in range(S)])
        z = np.exp(lls - L)
        se = z.std(ddof=1) / np.sqrt(S)
        assert abs(z.mean() - 1.0) < 4 * se + 1e-3, (th, z.mean(), se)


def test_particle_filter_unbiased_for_fsp_likelihood():
    check_filter_unbiased(fsp)


def test_gene_expression_filter_unbiased_against_fsp(S=300):
    """The gene-expression filter (the bench's network) against its exact
    likelihood: on the first 8 observation times the FSP box 0..16 x 0..250
    holds all but ~1e-12 of the mass, and mean exp(ll_PF - L_FSP) = 1."""
    w = W.gene_expression()
    y = w.observations()[:1, :8]
    times = w.obs_times[:8]
    for th in [w.theta_star, np.array([0.2, 0.1, 1.5, 0.02])]:
        L, leak = fsp.loglik(w.net, th, w.x0, [16, 250], times, y[0], w.C, w.sigma)
        assert abs(leak) < 1e-10
        lls = np.array([pf_oracle.pf_loglik(w.net, [th], w.x0, times, y, w.C, w.sigma, 200,
                                            700 + s)["loglik"][0] for s in range(S)])
        z = np.exp(lls - L)
        se = z.std(ddof=1) / np.sqrt(S)
        assert abs(z.mean() - 1.0) < 4 * se + 1e-3, (th, z.mean(), se)
        assert lls.mean() <= L + 4 * lls.std(ddof=1) / np.sqrt(S)


# A network of the cascade's kind small enough for an exact likelihood: three
# species, reactions of order 0, 1 and 2 (a heterodimer A + B and a homodimer
# B + B), two reactions sharing one rate column, two observed species.
THREE = {"reactants": np.array([[0, 0, 0], [1, 0, 0], [1, 1, 0], [0, 2, 0], [0, 0, 1], [0, 0, 1]],
                               np.int32),
         "products": np.array([[1, 0, 0], [0, 1, 0], [0, 0, 1], [0, 0, 0], [0, 0, 0], [1, 0, 0]],
                              np.int32),
         "rate_index": np.array([0, 1, 2, 3, 4, 4], np.int32)}


def test_second_order_network_filter_unbiased_against_fsp(S=300):
    """The filter oracle on THREE (the features of the 10-species cascade,
    whose own likelihood has no FSP box): on the box 0..25^3 the FSP
    likelihood loses < 1e-10 of the mass, and mean exp(ll_PF - L_FSP) = 1 at
    the data-generating theta and at a perturbed one; Jensen for the mean of
    ll."""
    th_star = np.array([2.0, 0.6, 0.15, 0.1, 0.25])
    x0 = np.array([2, 1, 0], np.int32)
    times = np.arange(1.0, 7.0)
    C = np.array([[1.0, 0.0, 0.0], [0.0, 0.0, 1.0]])
    sigma = np.array([1.0, 1.5])
    path, _, _ = pf_oracle.ssa_paths(THREE, th_star, x0, times, 1, seed=5)
    y = (path[0] @ C.T + np.random.default_rng(9).normal(size=(len(times), 2)) * sigma)[None]
    for th in [th_star, th_star * np.array([1.5, 0.7, 1.0, 2.0, 0.8])]:
        L, leak = fsp.loglik(THREE, th, x0, [25, 25, 25], times, y[0], C, sigma)
        assert abs(leak) < 1e-10
        lls = np.array([pf_oracle.pf_loglik(THREE, [th], x0, times, y, C, sigma, 200,
                                            900 + s)["loglik"][0] for s in range(S)])
        z = np.exp(lls - L)
        se = z.std(ddof=1) / np.sqrt(S)
        assert abs(z.mean() - 1.0) < 4 * se + 1e-3, (th, z.mean(), se)
        assert lls.mean() <= L + 4 * lls.std(ddof=1) / np.sqrt(S)


# ------------------------------------------------------------- mutants ----
MUTANTS = {
    "propagate_transposed": ("splinalg.expm_multiply(Q.T.tocsc() * dt, alpha)",
                             "splinalg.expm_multiply(Q.tocsc() * dt, alpha)", "telegraph"),
    "variance_not_squared": ("var = np.broadcast_to(sigma ** 2, mean.shape).copy()",
                             "var = np.broadcast_to(sigma, mean.shape).copy()", "birth_death"),
    "no_diagonal": ("vals.append(-A.sum(axis=1))", "vals.append(0.0 * A.sum(axis=1))",
                    "telegraph"),
    "strides_off_by_one": ("st[u] = st[u + 1] * (box_max[u + 1] + 1)",
                           "st[u] = st[u + 1] * box_max[u + 1]", "telegraph"),
    "power_law_dimer": ("h[:, r] *= X[:, u] * (X[:, u] - 1) // 2", "h[:, r] *= X[:, u] * X[:, u]",
                        "second_order"),
    "no_normalisation": ("alpha = w / c", "alpha = w", "filter"),
}
CHECKS = {
    "birth_death": check_birth_death_closed_form,
    "telegraph": check_telegraph_moments,
    "second_order": lambda f: check_second_order_law(f, n=8000),
    "filter": lambda f: check_filter_unbiased(f, S=120),
}


def variant(old, new):
    import inspect
    src = inspect.getsource(fsp)
    assert src.count(old) == 1, old
    mod = types.ModuleType("fsp_variant")
    exec(compile(src.replace(old, new), "fsp_variant", "exec"), mod.__dict__)
    return mod


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_fsp_pin_detects_mutant(name):
    old, new, check = MUTANTS[name]
    with pytest.raises((AssertionError, FloatingPointError, ValueError)):
        CHECKS[check](variant(old, new))
