"""Argument checks of the C ABI that run on the host before any device call
(CPU only): each malformed call returns PF_EINVAL with a message, so a caller
learns of the mistake without a GPU and without a launch."""
from __future__ import annotations

import shutil
from pathlib import Path

import numpy as np
import pytest

from paper_1606_08281_gb300 import workloads as W


@pytest.fixture(scope="module")
def pf():
    if shutil.which("nvcc") is None and not Path("/usr/local/cuda/bin/nvcc").exists():
        pytest.skip("nvcc not available")
    from paper_1606_08281_gb300 import build, pf as pfmod
    build.build()
    pfmod.load()
    return pfmod


def einval(pf, fn, *args, **kw):
    with pytest.raises(pf.PfError) as e:
        fn(*args, **kw)
    assert e.value.code == pf.PF_EINVAL, e.value
    return str(e.value)


def test_filter_arguments(pf):
    w = W.gene_expression().subset(T=2, K=6)
    th, y = w.thetas(3), w.observations()
    call = lambda **kw: pf.pf_loglik(  # noqa: E731
        kw.pop("net", w.net), kw.pop("th", th), w.x0, kw.pop("times", w.obs_times), kw.pop("y", y),
        w.C, kw.pop("sigma", w.sigma), kw.pop("N", 100), 1, **kw)
    assert "n_particles" in einval(pf, call, N=0)
    einval(pf, call, N=pf.PF_MAX_PARTICLES + 1 if hasattr(pf, "PF_MAX_PARTICLES") else 16385)
    assert "obs_times" in einval(pf, call, times=w.obs_times[::-1].copy())
    einval(pf, call, times=np.array([0.0, 1.0, 1.0, 2.0, 3.0, 4.0]))      # not strictly increasing
    einval(pf, call, times=np.array([-1.0, 1.0, 2.0, 3.0, 4.0, 5.0]))     # negative
    einval(pf, call, sigma=np.array([0.0]))
    einval(pf, call, event_budget=1 << 33)
    assert "block_threads" in einval(pf, call, block_threads=48)
    einval(pf, call, block_threads=256)
    einval(pf, call, net={"reactants": [[3, 0]], "products": [[0, 0]], "rate_index": None},
           th=np.ones((3, 1)))                                             # order 3 in one species


def test_cluster_arguments(pf):
    w = W.birth_death()
    call = lambda cb, N=64: pf.pf_loglik(  # noqa: E731
        w.net, w.thetas(2), w.x0, w.obs_times, w.observations(), w.C, w.sigma, N, 5,
        cluster_blocks=cb)
    assert "cluster_blocks" in einval(pf, call, -1)
    einval(pf, call, pf.PF_MAX_CLUSTER_BLOCKS + 1)
    # ceil(N / C) per block must leave the last block at least one particle
    for N, cb in [(6, 5), (9, 8), (2, 3), (1, 2)]:
        assert "empty" in einval(pf, call, cb, N)


def test_fsp_and_ode_arguments(pf):
    t = W.telegraph()
    einval(pf, pf.pf_fsp_loglik, t.net, t.thetas(2), t.x0, [1, 1, 5000], t.obs_times,
           t.observations(), t.C, t.sigma)                                  # box too large
    einval(pf, pf.pf_fsp_loglik, t.net, t.thetas(2), t.x0, [1, 1, -1], t.obs_times,
           t.observations(), t.C, t.sigma)
    e = W.erk()
    y = e.observations()
    einval(pf, pf.pf_erk_loglik, e.thetas(2), e.patterns, np.r_[0.0, e.obs_times[1:]], y)
    einval(pf, pf.pf_erk_loglik, e.thetas(2), e.patterns, e.obs_times, y, rtol=2.0)
    einval(pf, pf.pf_erk_loglik, e.thetas(2), e.patterns, e.obs_times, y, rtol=1e-10, atol=-1.0)


def test_batch_split_rule_and_cluster_share():
    """Host rules of the batch engine's cluster split: a request splits when
    its filters cannot fill one resident wave, and only if each block's share
    of the population fits the context's cluster arena (the bytes
    pf_ctx_config documents: ceil(N/C) (12 + 8U) + 16, plus 1 KB)."""
    from paper_1606_08281_gb300 import autotune, pf
    assert autotune.split_rule(152 * 4 - 1) and not autotune.split_rule(152 * 4)
    arena = pf.PF_CTX_CLUSTER_ARENA
    for N, C, U in [(4096, 2, 10), (4096, 4, 10), (200, 4, 9), (3, 4, 1), (4, 4, 1), (1000, 8, 16)]:
        share = -(-N // C)
        fits = N - (C - 1) * share >= 1 and share * (12 + 8 * U) + 16 + 1024 <= arena
        assert pf.split_fits(N, C, U) == fits, (N, C, U)
    assert not pf.split_fits(4096, 2, 10) and pf.split_fits(4096, 4, 10)
    assert not pf.split_fits(3, 4, 1)       # a block would hold no particle


def test_batch_tuner_coordinate_descent_and_cache(monkeypatch, tmp_path):
    """tune_batch's host logic with the context calls faked: it times every
    block-size pair, then the other cluster size (only when the mix has split
    requests) and the other grab, keeps the fastest, and a second call with the
    same mix signature comes from the cache without timing anything."""
    from paper_1606_08281_gb300 import autotune, pf
    cost = {(64, 128): 1.0, (128, 128): 2.0, (64, 64): 3.0, (128, 64): 4.0}
    made = []

    def fake_create(budget, slots, max_particles, block_threads, cluster_blocks, grab):
        made.append((tuple(block_threads), cluster_blocks, grab))
        return len(made)

    monkeypatch.setattr(pf, "pf_ctx_create_config", fake_create)
    monkeypatch.setattr(pf, "pf_ctx_destroy", lambda c: None)
    clock = {"t": 0.0}
    monkeypatch.setattr(pf, "pf_ctx_run_batch", lambda c, reqs: clock.__setitem__(
        "t", clock["t"] + reqs[0]))
    monkeypatch.setattr(autotune.time, "perf_counter", lambda: clock["t"])

    def make(ctx, ids, frac, cluster):
        bt, cb, gr = made[ctx - 1]
        t = cost[(bt[0], bt[1])] + (0.5 if cb == 2 else 0.0) - (0.25 if gr == 4 else 0.0)
        return [t * frac / 0.125]

    shapes = [("gene_expression", 64, 1000, 50, True)]
    cache = tmp_path / "tune.json"
    cfg = autotune.tune_batch(make, shapes, cache=cache, load_problems=lambda c: {})
    assert cfg["block_threads"] == [64, 128, 128, 128]
    assert cfg["cluster_blocks"] == 4 and cfg["grab"] == 4
    assert len(cfg["timings_s"]) == 6          # 4 block pairs, cluster 2, grab 4
    n = len(made)
    again = autotune.tune_batch(make, shapes, cache=cache, load_problems=lambda c: {})
    assert again == cfg and len(made) == n
    # no split request: the cluster size is not tried
    made.clear()
    cfg2 = autotune.tune_batch(make, [("cascade", 8, 512, 100, False)], cache=None,
                               load_problems=lambda c: {})
    assert not any(k.startswith("cluster") for k in cfg2["timings_s"])


def test_heterogeneous_mix_composition():
    """The batched-launch mix: 64 seeded requests over the three networks with
    theta counts, particle counts and observation prefixes in their stated
    ranges, plus one Lac-Gfp request of the workload's first 32 rows; the same
    seed gives the same mix."""
    mix = W.hetero_mix()
    assert len(mix) == 65
    lac = [s for s in mix if s.problem == "lac_gfp"]
    assert len(lac) == 1 and len(lac[0].thetas) == 32 and lac[0].n_particles == 200
    assert np.array_equal(lac[0].thetas, W.lac_gfp().thetas(32))
    for s in mix[:-1]:
        assert s.problem in ("birth_death", "gene_expression", "cascade")
        assert 1 <= len(s.thetas) <= 4096
        assert s.n_particles in (256, 512, 1024, 2048, 4096)
        assert 10 <= s.K_use <= 100 and s.K_use <= W.get(s.problem).K
    again = W.hetero_mix()
    assert all(np.array_equal(a.thetas, b.thetas) and a.seed == b.seed for a, b in zip(mix, again))
    small = W.hetero_mix(n_requests=48, max_theta_cascade=64)
    assert all(len(s.thetas) <= 64 for s in small if s.problem == "cascade")
