"""Parity of the model extensions (pf_model: composed rates, uniform random
initial counts, offset mean and state-dependent observation variance, the
forms of the paper's Lac-Gfp example) between the CUDA path and the oracle.

Same bar as test_gpu_parity: per filter, fired reactions and the history
digest bit-identical, final states identical, log-likelihoods within 1e-9
relative.  With a state-dependent variance each log-weight holds a log(v):
CUDA's and glibc's logarithms may differ in the last place, which moves the
likelihood by ~1e-16 relative and the resampling draws only if a log-weight
sits within that distance of a 2^-20 grid boundary (the integer weights use
the rounded log-weights), i.e. never at these sizes.
"""
from __future__ import annotations

import numpy as np
import pytest

from oracle import pf_oracle
from paper_1606_08281_gb300 import workloads as W

pytestmark = pytest.mark.gpu

RTOL = 1e-9
BD_MODEL = {"rate_coef": [[1.0, 3.0, 0.0], [0.0, 0.0, 1.0]], "x0_hi": [15], "obs_offset": [2.0],
            "obs_var": [[0.5]]}


@pytest.fixture(scope="module")
def pf():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1606_08281_gb300 import build, pf as pfmod
    build.build()
    pfmod.load()
    return pfmod


def run_both(pf, net, thetas, x0, times, y, C, sigma, N, seed, model, final_states=True, **kw):
    g = pf.pf_loglik(net, thetas, x0, times, y, C, sigma, N, seed, diagnostics=True,
                     final_states=final_states, model=model, **kw)
    o = pf_oracle.pf_loglik(net, thetas, x0, times, y, C, sigma, N, seed,
                            want_final_states=final_states, model=model)
    return g, o


def assert_parity(g, o, final_states=True):
    assert (g["status"] == o["status"]).all(), (g["status"], o["status"])
    ok = o["status"] == 0
    bad = np.argwhere(~((g["events"] == o["events"]) & (g["digest"] == o["digest"]))[ok])
    assert len(bad) == 0, f"history mismatch in filters {bad[:10].tolist()}"
    np.testing.assert_allclose(g["ll_traj"][ok], o["ll_traj"][ok], rtol=RTOL, atol=0)
    np.testing.assert_allclose(g["loglik"][ok], o["loglik"][ok], rtol=RTOL, atol=0)
    if final_states:
        assert (g["final_states"][ok] == o["final_states"][ok]).all()


def bd_problem(T=3):
    w = W.birth_death()
    rng = np.random.default_rng(11)
    ys = []
    for traj in range(T):
        xs, _, _ = pf_oracle.ssa_paths(W.birth_death_network(), [10.0, 0.2], [9], w.obs_times, 1,
                                       seed=700 + traj)
        xk = xs[0, :, 0].astype(float)
        ys.append(2.0 + 1.5 * xk + rng.normal(size=len(xk)) * np.sqrt(1.0 + 0.5 * xk))
    y = np.array(ys)[:, :, None]
    th = W.log_uniform(np.random.default_rng(12), [1.0, 0.1, 0.05], [20.0, 5.0, 1.0], 13)
    return w, th, y


@pytest.mark.parametrize("N", [1, 37, 200, 1000])
def test_birth_death_extended_model(pf, N):
    w, th, y = bd_problem()
    g, o = run_both(pf, W.birth_death_network(), th, [5], w.obs_times, y, [[1.5]], [1.0], N, 21,
                    BD_MODEL)
    assert_parity(g, o)


@pytest.mark.parametrize("part", ["rate_coef", "x0_hi", "obs_offset", "obs_var"])
def test_each_extension_alone(pf, part):
    w, th, y = bd_problem(T=2)
    model = {part: BD_MODEL[part]}
    if part == "rate_coef":
        thetas = th
    else:
        thetas = th[:, [0, 2]] * np.array([4.0, 1.0])         # plain rates k1, k2
    g, o = run_both(pf, W.birth_death_network(), thetas, [5], w.obs_times, y, [[1.5]], [1.0],
                    64, 5, model)
    assert_parity(g, o)


def test_degenerate_extensions_equal_basic_model(pf):
    """x0_hi == x0 and a zero offset leave the basic path's results bit for bit."""
    w = W.gene_expression().subset(T=2, K=8)
    th = w.thetas(6)
    base = pf.pf_loglik(w.net, th, w.x0, w.obs_times, w.observations(), w.C, w.sigma, 100, 3,
                        diagnostics=True)
    ext = pf.pf_loglik(w.net, th, w.x0, w.obs_times, w.observations(), w.C, w.sigma, 100, 3,
                       diagnostics=True, model={"x0_hi": w.x0, "obs_offset": [0.0],
                                                "rate_coef": np.eye(4)})
    assert (base["digest"] == ext["digest"]).all()
    assert (base["loglik"] == ext["loglik"]).all()


def test_lac_gfp_subset(pf):
    """The Lac-Gfp network (9 species, 18 reactions, composed rate, shared
    rate, uniform initial counts, fluorescence observation with background)."""
    w = W.lac_gfp()
    th = np.vstack([w.theta_star, w.thetas(5)])
    y = w.observations()[:2, :4]
    g, o = run_both(pf, w.net, th, w.x0, w.obs_times[:4], y, w.C, w.sigma, 48, w.filter_seed,
                    w.model)
    assert_parity(g, o)
    assert int(g["events"].sum()) > 10**5


def test_lac_gfp_global_memory_population(pf):
    """A population too large for shared memory runs from the global slab."""
    w = W.lac_gfp()
    th = w.theta_star[None, :]
    y = w.observations()[:1, :2]
    g, o = run_both(pf, w.net, th, w.x0, w.obs_times[:2], y, w.C, w.sigma, 5000, 9, w.model,
                    final_states=False)
    assert_parity(g, o, final_states=False)


def test_lac_gfp_in_batch_context(pf):
    """A context loaded with pf_ctx_load_problem_model returns the plain call's values."""
    w = W.lac_gfp()
    ctx = pf.pf_ctx_create(mem_budget_bytes=0, n_slots=2, max_particles=1024)
    try:
        pid = pf.pf_ctx_load_problem(ctx, w.net, 18, w.x0, w.obs_times, w.observations(), w.C,
                                     w.sigma, model=w.model)
        th = w.thetas(4)
        req = pf.Request(pid, th, 64, 17, K_use=3)
        pf.pf_ctx_run_batch(ctx, [req])
        ref = pf.pf_loglik(w.net, th, w.x0, w.obs_times[:3], w.observations()[:, :3], w.C,
                           w.sigma, 64, 17, model=w.model)
        assert (req.status == ref["status"]).all()
        assert np.array_equal(req.loglik, ref["loglik"])
    finally:
        pf.pf_ctx_destroy(ctx)


def test_early_rejection_with_state_dependent_variance(pf):
    """The level-set bound stays an upper bound (v_p >= sigma_p^2): rows not
    rejected keep their full values, rejected rows are below the threshold."""
    w, th, y = bd_problem()
    full = pf.pf_loglik(W.birth_death_network(), th, [5], w.obs_times, y, [[1.5]], [1.0], 80, 4,
                        model=BD_MODEL)
    thr = float(np.median(full["loglik"]))
    r = pf.pf_loglik(W.birth_death_network(), th, [5], w.obs_times, y, [[1.5]], [1.0], 80, 4,
                     model=BD_MODEL, reject_below=thr)
    rej = r["status"] == pf.PF_ST_REJECTED
    assert (full["loglik"][rej] < thr).all()
    assert np.array_equal(r["loglik"][~rej], full["loglik"][~rej])


@pytest.mark.parametrize("bad", [
    {"obs_var": [[-1.0]]}, {"x0_hi": [2]}, {"rate_coef": [[1.0, -1.0, 0.0], [0.0, 0.0, 1.0]]},
    {"obs_offset": [np.inf]}])
def test_invalid_model_rejected(pf, bad):
    w, th, y = bd_problem(T=1)
    with pytest.raises(pf.PfError) as e:
        pf.pf_loglik(W.birth_death_network(), th, [5], w.obs_times, y, [[1.5]], [1.0], 10, 1,
                     model=bad)
    assert e.value.code == pf.PF_EINVAL


def test_too_many_rate_terms_rejected(pf):
    w, th, y = bd_problem(T=1)
    with pytest.raises(pf.PfError):
        pf.pf_loglik(W.birth_death_network(), np.ones((2, 6)), [5], w.obs_times, y, [[1.5]],
                     [1.0], 10, 1, model={"rate_coef": np.ones((2, 6))})
