"""Batching and serving through the C ABI context (pf_ctx_*).

A request's result depends only on its own inputs, so every request in a
batch -- whatever else shares the launch -- must equal the plain pf_loglik
call with the same problem, theta, N, observation prefix and seed, bit for
bit.  Requests mix problems, theta counts, particle counts (shared-memory and
global-memory populations) and observation prefixes.
"""
from __future__ import annotations

import numpy as np
import pytest

from paper_1606_08281_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pf():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1606_08281_gb300 import build, pf as pfmod
    build.build()
    pfmod.load()
    return pfmod


@pytest.fixture(scope="module")
def ctx(pf):
    c = pf.pf_ctx_create(mem_budget_bytes=0, n_slots=3, max_particles=4096)
    yield c
    pf.pf_ctx_destroy(c)


@pytest.fixture(scope="module")
def problems(pf, ctx):
    out = {}
    for name in ("birth_death", "gene_expression", "cascade"):
        w = W.get(name)
        d = w.R
        pid = pf.pf_ctx_load_problem(ctx, w.net, d, w.x0, w.obs_times, w.observations(), w.C,
                                     w.sigma)
        out[name] = (pid, w)
    return out


def plain(pf, w, th, N, seed, K):
    return pf.pf_loglik(w.net, th, w.x0, w.obs_times[:K], w.observations()[:, :K, :], w.C,
                        w.sigma, N, seed)


SPECS = [  # (problem, M, N, K, seed)
    ("birth_death", 37, 100, 20, 11),
    ("gene_expression", 9, 1000, 12, 12),        # population in the small arena (4 blocks/SM)
    ("gene_expression", 3, 2048, 6, 13),         # population in the large arena (2 blocks/SM)
    ("cascade", 2, 256, 4, 14),
    ("cascade", 1, 600, 3, 15),                  # cascade in the large arena
    ("cascade", 1, 2048, 3, 18),                 # cascade in a global slab (106 KB)
    ("birth_death", 1, 1, 5, 16),                # a single particle
    ("gene_expression", 0, 64, 5, 17),           # an empty request
]


def make_requests(pf, problems, specs):
    reqs = []
    for name, M, N, K, seed in specs:
        pid, w = problems[name]
        th = W.log_uniform(np.random.default_rng(seed), w.prior_lo, w.prior_hi, max(M, 0))
        reqs.append((pf.Request(pid, th, N, seed, K_use=K), w, th, N, seed, K))
    return reqs


def test_batch_matches_plain_calls(pf, ctx, problems):
    reqs = make_requests(pf, problems, SPECS)
    pf.pf_ctx_run_batch(ctx, [r[0] for r in reqs])
    for r, w, th, N, seed, K in reqs:
        ref = plain(pf, w, th, N, seed, K)
        assert (r.status == ref["status"]).all()
        assert np.array_equal(r.loglik, ref["loglik"]), (w.name, N, K)


def test_result_alone_equals_result_in_the_mix(pf, ctx, problems):
    reqs = make_requests(pf, problems, SPECS)
    target = reqs[1]
    alone = make_requests(pf, problems, [SPECS[1]])[0]
    pf.pf_ctx_run_batch(ctx, [alone[0]])
    pf.pf_ctx_run_batch(ctx, [r[0] for r in reqs])
    assert np.array_equal(alone[0].loglik, target[0].loglik)


def test_serving_submit_and_poll(pf, ctx, problems):
    specs = [SPECS[i % 5] for i in range(12)]
    specs = [(n, M, N, K, 100 + i) for i, (n, M, N, K, _) in enumerate(specs)]
    reqs = make_requests(pf, problems, specs)
    for r in reqs:
        pf.pf_submit(ctx, r[0])
    for r, w, th, N, seed, K in reqs:
        while not pf.pf_poll(ctx, r, wait_ms=1000):
            pass
        ref = plain(pf, w, th, N, seed, K)
        assert np.array_equal(r.loglik, ref["loglik"])
        assert r.t_done >= r.t_submit
    st = pf.pf_ctx_stats(ctx)
    assert st["requests"] >= len(reqs) and st["batches"] >= 1


def test_admission_by_memory_budget(pf, problems):
    """A small budget admits requests a few at a time; all still finish with the
    right results, and a request larger than the budget is refused."""
    small = pf.pf_ctx_create(mem_budget_bytes=40_000, n_slots=2, max_particles=1024)
    try:
        pids = {}
        for name in ("birth_death", "gene_expression"):
            w = W.get(name)
            pids[name] = pf.pf_ctx_load_problem(small, w.net, w.R, w.x0, w.obs_times,
                                                w.observations(), w.C, w.sigma)
        probs = {k: (pids[k], W.get(k)) for k in pids}
        specs = [("birth_death", 40, 100, 20, 200 + i) for i in range(6)]
        specs += [("gene_expression", 8, 200, 5, 300 + i) for i in range(3)]
        reqs = make_requests(pf, probs, specs)
        for r in reqs:
            pf.pf_submit(small, r[0])
        for r, w, th, N, seed, K in reqs:
            while not pf.pf_poll(small, r, wait_ms=1000):
                pass
            assert np.array_equal(r.loglik, plain(pf, w, th, N, seed, K)["loglik"])
        assert pf.pf_ctx_stats(small)["batches"] >= 3
        big = make_requests(pf, probs, [("gene_expression", 4000, 64, 5, 1)])[0][0]
        with pytest.raises(pf.PfError) as e:
            pf.pf_submit(small, big)
        assert e.value.code == pf.PF_EBUSY
    finally:
        pf.pf_ctx_destroy(small)


def test_bad_requests(pf, ctx, problems):
    pid, w = problems["birth_death"]
    with pytest.raises(pf.PfError) as e:
        pf.pf_submit(ctx, pf.Request(99, np.ones((1, 2)), 10, 1))
    assert e.value.code == pf.PF_ENOTFOUND
    with pytest.raises(pf.PfError):
        pf.pf_submit(ctx, pf.Request(pid, np.ones((1, 2)), 10, 1, K_use=999))
    with pytest.raises(pf.PfError):
        pf.pf_submit(ctx, pf.Request(pid, np.ones((1, 2)), 100000, 1))


def test_batch_early_rejection_matches_plain(pf, ctx, problems):
    """Requests carrying a level-set threshold: the context rejects exactly the
    rows the plain call rejects, and keeps the others' values."""
    pid, w = problems["gene_expression"]
    th = W.log_uniform(np.random.default_rng(77), w.prior_lo, w.prior_hi, 40)
    full = plain(pf, w, th, 200, 5, 10)
    thr = float(np.median(full["loglik"]))
    reqs = [pf.Request(pid, th, 200, 5, K_use=10, loglik_threshold=thr),
            pf.Request(problems["birth_death"][0], problems["birth_death"][1].thetas(8), 50, 6)]
    pf.pf_ctx_run_batch(ctx, reqs)
    ref = pf.pf_loglik(w.net, th, w.x0, w.obs_times[:10], w.observations()[:, :10, :], w.C,
                       w.sigma, 200, 5, reject_below=thr)
    assert (reqs[0].status == ref["status"]).all()
    assert np.array_equal(reqs[0].loglik, ref["loglik"])
    assert (reqs[0].status == pf.PF_ST_REJECTED).sum() == (full["loglik"] < thr).sum()


def test_batch_covers_every_tier(pf):
    """Requests on networks of every kernel group (reaction tiers with state
    in registers or in shared memory; populations in the small and the large
    arena and in a global slab) in one batch equal their plain calls bit for
    bit."""
    from test_gpu_parity import tier_problem
    c = pf.pf_ctx_create(mem_budget_bytes=0, n_slots=2, max_particles=8192)
    try:
        reqs = []
        for i, (kind, N) in enumerate([("r4_u5", 128), ("r8_u4", 128), ("r8_u6", 256),
                                       ("r15_u8", 128), ("r15_u8", 6000)]):
            net, th, x0, times, y, C, sigma = tier_problem(kind)
            pid = pf.pf_ctx_load_problem(c, net, th.shape[1], x0, times, y, C, sigma)
            reqs.append((pf.Request(pid, th[:3], N, 50 + i), net, th[:3], x0, times, y, C, sigma, N,
                         50 + i))
        pf.pf_ctx_run_batch(c, [r[0] for r in reqs])
        for r, net, th, x0, times, y, C, sigma, N, seed in reqs:
            ref = pf.pf_loglik(net, th, x0, times, y, C, sigma, N, seed)
            assert (r.status == ref["status"]).all()
            assert np.array_equal(r.loglik, ref["loglik"]), (N, r.loglik, ref["loglik"])
    finally:
        pf.pf_ctx_destroy(c)


def oracle_rows(w, th, N, seed, K, ids=None):
    from oracle import pf_oracle
    return pf_oracle.pf_loglik(w.net, th, w.x0, w.obs_times[:K], w.observations()[:, :K, :], w.C,
                               w.sigma, N, seed, theta_ids=ids)


def test_batch_matches_the_oracle(pf, ctx, problems):
    """The context's results against the oracle directly (not only against
    pf_loglik): every network, populations in both shared-memory arenas,
    requests with theta id bases."""
    specs = [("birth_death", 25, 100, 20, 61, 0), ("gene_expression", 6, 1000, 10, 62, 500),
             ("gene_expression", 2, 2048, 5, 63, 0), ("cascade", 2, 256, 4, 64, 9000)]
    reqs = []
    for name, M, N, K, seed, base in specs:
        pid, w = problems[name]
        th = W.log_uniform(np.random.default_rng(seed), w.prior_lo, w.prior_hi, M)
        reqs.append((pf.Request(pid, th, N, seed, K_use=K, theta_id_base=base), w, th, N, seed, K,
                     base))
    pf.pf_ctx_run_batch(ctx, [r[0] for r in reqs])
    for r, w, th, N, seed, K, base in reqs:
        o = oracle_rows(w, th, N, seed, K, ids=np.arange(base, base + len(th)))
        assert (r.status == o["status"]).all(), w.name
        np.testing.assert_allclose(r.loglik, o["loglik"], rtol=1e-9, atol=0)


def rejection_threshold(values: np.ndarray) -> float:
    """A threshold between two neighbouring values near the median, so that no
    value lies within rounding of it (the decision is then exact)."""
    v = np.sort(values[np.isfinite(values)])
    i = len(v) // 2
    gaps = np.diff(v[max(0, i - 5): i + 6])
    j = max(0, i - 5) + int(np.argmax(gaps))
    return float(0.5 * (v[j] + v[j + 1]))


def test_early_rejection_decisions_against_the_oracle(pf, ctx, problems):
    """REJECTED exactly for the rows whose full oracle log-likelihood is below
    the threshold (Alg. 2 keeps theta only if l_hat >= epsilon); every other
    row equals the oracle's value.  Plain call and batch request."""
    pid, w = problems["gene_expression"]
    th = W.log_uniform(np.random.default_rng(91), w.prior_lo, w.prior_hi, 48)
    N, seed, K = 200, 19, 12
    o = oracle_rows(w, th, N, seed, K)
    thr = rejection_threshold(o["loglik"])
    below = o["loglik"] < thr
    assert 10 < below.sum() < 38
    plain_cut = pf.pf_loglik(w.net, th, w.x0, w.obs_times[:K], w.observations()[:, :K, :], w.C,
                             w.sigma, N, seed, reject_below=thr)
    req = pf.Request(pid, th, N, seed, K_use=K, loglik_threshold=thr)
    pf.pf_ctx_run_batch(ctx, [req])
    for st, ll in ((plain_cut["status"], plain_cut["loglik"]), (req.status, req.loglik)):
        assert (st[below] == pf.PF_ST_REJECTED).all()
        assert (st[~below] == 0).all()
        np.testing.assert_allclose(ll[~below], o["loglik"][~below], rtol=1e-9, atol=0)
        assert np.isneginf(ll[below]).all()


def test_launch_shape_and_cluster_split(pf):
    """A context with its own launch shape (threads per block for each tier,
    two filters per work-list grab, 4-block clusters): requests run one block
    per filter equal their plain calls bit for bit whatever the shape; requests
    asking to be split equal pf_loglik with the same cluster size and the
    oracle; a Lac-Gfp request (model extensions) split in the mix too."""
    from oracle import pf_oracle
    c = pf.pf_ctx_create_config(0, 2, 4096, block_threads=(64, 96, 128, 96), cluster_blocks=4,
                                grab=2)
    try:
        names = ("birth_death", "gene_expression", "cascade", "lac_gfp")
        wl = {n: W.get(n) for n in names}
        pids = {n: pf.pf_ctx_load_problem(c, wl[n].net, len(wl[n].prior_lo), wl[n].x0,
                                          wl[n].obs_times, wl[n].observations(), wl[n].C,
                                          wl[n].sigma, model=wl[n].model) for n in names}
        specs = [("birth_death", 30, 100, 20, 71, 0), ("gene_expression", 5, 1000, 8, 72, 4),
                 ("cascade", 2, 512, 4, 73, 4), ("lac_gfp", 3, 200, 4, 74, 4),
                 ("gene_expression", 4, 600, 6, 75, 0)]
        reqs = []
        for name, M, N, K, seed, C in specs:
            w = wl[name]
            # Lac-Gfp: the workload's first rows (its prior's tail holds filters
            # of 10^9 reactions, beyond the oracle in a test)
            th = (w.thetas(M) if name == "lac_gfp" else
                  W.log_uniform(np.random.default_rng(seed), w.prior_lo, w.prior_hi, M))
            reqs.append((pf.Request(pids[name], th, N, seed, K_use=K, cluster_blocks=C), w, th, N,
                         seed, K, C))
        pf.pf_ctx_run_batch(c, [r[0] for r in reqs])
        for r, w, th, N, seed, K, C in reqs:
            ref = pf.pf_loglik(w.net, th, w.x0, w.obs_times[:K], w.observations()[:, :K, :], w.C,
                               w.sigma, N, seed, model=w.model, cluster_blocks=C)
            assert (r.status == ref["status"]).all(), w.name
            assert np.array_equal(r.loglik, ref["loglik"]), (w.name, C)
            o = pf_oracle.pf_loglik(w.net, th, w.x0, w.obs_times[:K], w.observations()[:, :K, :],
                                    w.C, w.sigma, N, seed, model=w.model)
            ok = o["status"] == 0
            assert (r.status == o["status"]).all()
            np.testing.assert_allclose(r.loglik[ok], o["loglik"][ok], rtol=1e-9, atol=0)
        # a split request must use the context's cluster size
        with pytest.raises(pf.PfError) as e:
            pf.pf_submit(c, pf.Request(pids["gene_expression"], reqs[1][2], 600, 1, K_use=4,
                                       cluster_blocks=2))
        assert e.value.code == pf.PF_EINVAL
    finally:
        pf.pf_ctx_destroy(c)
    with pytest.raises(pf.PfError):
        pf.pf_ctx_create_config(0, 1, 1024, block_threads=(48, 0, 0, 0))
    with pytest.raises(pf.PfError):
        pf.pf_ctx_create_config(0, 1, 1024, cluster_blocks=9)


def test_many_batches_through_the_cluster_groups(pf):
    """Hundreds of graph replays of one context whose graph carries the
    cluster groups of every tier (most of them empty in a batch): every batch
    finishes, and a split request and a one-block request give the same bits
    in every replay.  Guards the cluster groups' exit (no block leaves while
    another still reads its shared memory) and the worker's completion path."""
    c = pf.pf_ctx_create_config(0, 3, 1024, cluster_blocks=4, grab=2)
    try:
        w = W.get("birth_death")
        pid = pf.pf_ctx_load_problem(c, w.net, len(w.prior_lo), w.x0, w.obs_times,
                                     w.observations(), w.C, w.sigma)
        th = W.log_uniform(np.random.default_rng(91), w.prior_lo, w.prior_hi, 3)
        first = None
        for i in range(400):
            reqs = [pf.Request(pid, th, 100, 5, K_use=6, cluster_blocks=4),
                    pf.Request(pid, th, 100, 5, K_use=6)]
            if i % 2:                        # the same requests by pf_submit / pf_poll
                for r in reqs:
                    pf.pf_submit(c, r)
                for r in reqs:
                    while not pf.pf_poll(c, r, wait_ms=1000):
                        pass
            else:
                pf.pf_ctx_run_batch(c, reqs)
            got = [r.loglik.copy() for r in reqs]
            if first is None:
                first = got
            for a, b in zip(got, first):
                assert np.array_equal(a, b), i
        assert pf.pf_ctx_stats(c)["batches"] >= 400
    finally:
        pf.pf_ctx_destroy(c)
