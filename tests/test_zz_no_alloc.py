"""The allocation-free entry point, pf_loglik_noalloc, through the C ABI.

Some callers cannot allocate device memory (their GPU memory is owned by
another allocator, or their request path cannot afford cudaMalloc).  This
entry point keeps its scratch in a fixed static device array.  Its results
must equal those of pf_loglik, on two calls in a row (the second call reuses
the array the first one left behind).  Kept in its own file, collected last.
"""
from __future__ import annotations

import numpy as np
import pytest

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


def _case(pf, w, M, N, seed):
    import torch
    dev = torch.device("cuda:0")
    th = w.thetas(M)
    ref = pf.pf_loglik(w.net, th, w.x0, w.obs_times, w.observations(), w.C, w.sigma, N, seed)
    th_d = torch.from_numpy(th).to(dev)
    y_d = torch.from_numpy(w.observations()).to(dev)
    ll = torch.full((M,), 123.0, dtype=torch.float64, device=dev)
    st = torch.full((M,), 255, dtype=torch.uint8, device=dev)
    pf.pf_loglik_noalloc(w.net, th_d, w.x0, w.obs_times, y_d, w.C, w.sigma, N, seed, ll, st)
    torch.cuda.synchronize()
    return ref, ll.cpu().numpy(), st.cpu().numpy()


def test_noalloc_matches_pf_loglik_on_two_calls_in_a_row(pf):
    # first call: gene expression subset; second call: a different network and size
    w1 = W.gene_expression().subset(T=3, K=10)
    ref, ll, st = _case(pf, w1, 40, 300, 17)
    np.testing.assert_allclose(ll, ref["loglik"], rtol=RTOL, atol=0)
    assert (st == ref["status"]).all()
    w2 = W.birth_death()
    ref, ll, st = _case(pf, w2, 25, 100, 18)
    np.testing.assert_allclose(ll, ref["loglik"], rtol=RTOL, atol=0)
    assert (st == ref["status"]).all()


def test_noalloc_rejects_problems_beyond_its_scratch(pf):
    """A problem whose scratch exceeds the fixed array is refused on the host
    (PF_EINVAL) before any device work."""
    import ctypes as ct

    import torch
    w = W.birth_death()
    dev = torch.device("cuda:0")
    th = torch.ones((8, 2), dtype=torch.float64, device=dev)
    y = torch.from_numpy(w.observations()).to(dev)
    ll = torch.empty(8, dtype=torch.float64, device=dev)
    n = pf._Net(w.net)
    ts = np.ascontiguousarray(w.obs_times)
    rc = pf.load().pf_loglik_noalloc(
        ct.byref(n.s), th.data_ptr(), 10**6, 2, pf._hptr(np.array([10], np.int32)),
        pf._hptr(ts), 20, y.data_ptr(), 4000, 1, pf._hptr(np.array([1.0])),
        pf._hptr(np.array([1.0])), 100, ct.c_uint64(1), ll.data_ptr(), None, ct.c_uint64(0),
        None)
    assert rc == pf.PF_EINVAL
    assert "scratch" in pf.pf_last_error()


def test_noalloc_refuses_populations_beyond_shared_memory(pf):
    """pf_loglik runs populations beyond shared memory from global slabs it
    allocates; the allocation-free entry point refuses them (PF_EINVAL) on
    the host, before any device work."""
    import ctypes as ct

    import torch
    w = W.gene_expression().subset(T=1, K=3)
    dev = torch.device("cuda:0")
    th = torch.from_numpy(w.thetas(2)).to(dev)
    y = torch.from_numpy(w.observations()).to(dev)
    ll = torch.empty(2, dtype=torch.float64, device=dev)
    n = pf._Net(w.net)
    ts = np.ascontiguousarray(w.obs_times)
    rc = pf.load().pf_loglik_noalloc(
        ct.byref(n.s), th.data_ptr(), 2, 4, pf._hptr(np.zeros(2, np.int32)), pf._hptr(ts), 3,
        y.data_ptr(), 1, 1, pf._hptr(np.ascontiguousarray(w.C)), pf._hptr(w.sigma), 16384,
        ct.c_uint64(1), ll.data_ptr(), None, ct.c_uint64(0), None)
    assert rc == pf.PF_EINVAL
    assert "shared memory" in pf.pf_last_error()


def test_noalloc_wrapper_checks_its_tensors(pf):
    """The binding refuses, without copying, tensors the call cannot read as
    they are: a wrong dtype, a non-contiguous view, a host tensor, a short
    output."""
    import torch
    w = W.birth_death()
    dev = torch.device("cuda:0")
    th = torch.from_numpy(w.thetas(8)).to(dev)
    y = torch.from_numpy(w.observations()).to(dev)
    ll = torch.empty(8, dtype=torch.float64, device=dev)
    args = (w.net, th, w.x0, w.obs_times, y, w.C, w.sigma, 64, 5)
    with pytest.raises(ValueError, match="float64"):
        pf.pf_loglik_noalloc(w.net, th.float(), w.x0, w.obs_times, y, w.C, w.sigma, 64, 5, ll)
    wide = torch.from_numpy(np.repeat(w.thetas(8), 2, axis=1)).to(dev)
    with pytest.raises(ValueError, match="contiguous"):
        pf.pf_loglik_noalloc(w.net, wide[:, ::2], w.x0, w.obs_times, y, w.C, w.sigma, 64, 5, ll)
    with pytest.raises(ValueError, match="CUDA"):
        pf.pf_loglik_noalloc(*args, ll.cpu())
    with pytest.raises(ValueError, match="elements"):
        pf.pf_loglik_noalloc(*args, ll[:4])
    with pytest.raises(ValueError, match="uint8"):
        pf.pf_loglik_noalloc(*args, ll, torch.empty(8, dtype=torch.int32, device=dev))
