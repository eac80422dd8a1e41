"""Theta ids in the random-number counter (pf_options.theta_ids,
pf_request.theta_id_base): a batch split over several calls or requests, or
a subset of its rows evaluated with their ids, reproduces the whole batch bit
for bit, and equals the oracle evaluated with the same ids."""
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


def call(pf, w, th, N, seed, **kw):
    return pf.pf_loglik(w.net, th, w.x0, w.obs_times, w.observations(), w.C, w.sigma, N, seed,
                        diagnostics=True, **kw)


@pytest.mark.parametrize("cluster", [0, 2])
def test_two_half_batches_equal_the_whole_batch(pf, cluster):
    w = W.gene_expression().subset(T=3, K=8)
    th = w.thetas(30)
    whole = call(pf, w, th, 200, 9, cluster_blocks=cluster)
    a = call(pf, w, th[:13], 200, 9, theta_ids=np.arange(13), cluster_blocks=cluster)
    b = call(pf, w, th[13:], 200, 9, theta_ids=np.arange(13, 30), cluster_blocks=cluster)
    for k in ("loglik", "digest", "events", "ll_traj"):
        assert np.array_equal(np.concatenate([a[k], b[k]]), whole[k]), k
    # without ids the second half is a different batch (ids restart at 0)
    c = call(pf, w, th[13:], 200, 9, cluster_blocks=cluster)
    assert not np.array_equal(c["digest"], whole["digest"][13:])


def test_scattered_rows_with_ids_match_the_oracle(pf):
    """Rows 3, 97, 250 and 4000 of a batch, evaluated alone with their ids,
    on the GPU (shared-memory and global-slab populations) and in the oracle."""
    w = W.gene_expression().subset(T=2, K=6)
    full = w.thetas()
    ids = np.array([3, 97, 250, 4000])
    for N in (300, 9800):
        g = call(pf, w, full[ids], N, 41, theta_ids=ids)
        o = pf_oracle.pf_loglik(w.net, full[ids], w.x0, w.obs_times, w.observations(), w.C,
                                w.sigma, N, 41, theta_ids=ids)
        assert (g["digest"] == o["digest"]).all() and (g["events"] == o["events"]).all()
        np.testing.assert_allclose(g["ll_traj"], o["ll_traj"], rtol=RTOL, atol=0)
        np.testing.assert_allclose(g["loglik"], o["loglik"], rtol=RTOL, atol=0)


def test_device_ids_equal_host_ids(pf):
    import torch
    w = W.birth_death()
    th = w.thetas(20)
    ids = np.arange(100, 120)
    h = call(pf, w, th, 64, 3, theta_ids=ids)
    dev = torch.device("cuda:0")
    d = pf.pf_loglik(w.net, torch.from_numpy(th).to(dev), w.x0, w.obs_times,
                     torch.from_numpy(w.observations()).to(dev), w.C, w.sigma, 64, 3,
                     diagnostics=True,
                     theta_ids=torch.from_numpy(ids.astype(np.int32)).to(dev))
    torch.cuda.synchronize()
    assert np.array_equal(d["loglik"].cpu().numpy(), h["loglik"])
    assert np.array_equal(d["digest"].cpu().numpy().view(np.uint64), h["digest"])


def test_request_split_with_id_bases_equals_one_request(pf):
    c = pf.pf_ctx_create(mem_budget_bytes=0, n_slots=2, max_particles=1024)
    try:
        w = W.gene_expression()
        pid = pf.pf_ctx_load_problem(c, w.net, w.R, w.x0, w.obs_times, w.observations(), w.C,
                                     w.sigma)
        th = w.thetas(50)
        whole = pf.Request(pid, th, 256, 77, K_use=8)
        pf.pf_ctx_run_batch(c, [whole])
        parts = [pf.Request(pid, th[:20], 256, 77, K_use=8),
                 pf.Request(pid, th[20:], 256, 77, K_use=8, theta_id_base=20)]
        pf.pf_ctx_run_batch(c, parts)
        assert np.array_equal(np.concatenate([parts[0].loglik, parts[1].loglik]), whole.loglik)
        # the same rows through pf_loglik with explicit ids
        ref = pf.pf_loglik(w.net, th[20:], w.x0, w.obs_times[:8], w.observations()[:, :8], w.C,
                           w.sigma, 256, 77, theta_ids=np.arange(20, 50))
        assert np.array_equal(parts[1].loglik, ref["loglik"])
        with pytest.raises(pf.PfError) as e:
            pf.pf_submit(c, pf.Request(pid, th[:2], 256, 1, theta_id_base=2**32 - 1))
        assert e.value.code == pf.PF_EINVAL
    finally:
        pf.pf_ctx_destroy(c)


def test_bad_theta_ids_are_refused_on_the_host(pf):
    w = W.birth_death()
    with pytest.raises(ValueError):
        call(pf, w, w.thetas(4), 16, 1, theta_ids=np.arange(3))
    with pytest.raises(ValueError):
        call(pf, w, w.thetas(2), 16, 1, theta_ids=np.array([-1, 0]))
