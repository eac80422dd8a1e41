"""The launch-parameter autotuner picks one of its candidates, caches it by
problem shape, and the tuned launch gives the same results as the default."""
from __future__ import annotations

import numpy as np
import pytest

from paper_1606_08281_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_autotune_caches_a_valid_choice(tmp_path):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1606_08281_gb300 import autotune, build, pf
    build.build()
    w = W.gene_expression().subset(T=2, K=5)
    cache = tmp_path / "tune.json"
    res = autotune.tune(w.net, w.thetas(64), w.x0, w.obs_times, w.observations(), w.C, w.sigma,
                        200, reps=1, sample_filters=128, cache=cache)
    assert res["block_threads"] in autotune.BLOCKS
    assert autotune.lookup(w.net, 200, w.K, w.T, cache=cache)["block_threads"] == res["block_threads"]
    a = pf.pf_loglik(w.net, w.thetas(16), w.x0, w.obs_times, w.observations(), w.C, w.sigma, 200, 3)
    b = pf.pf_loglik(w.net, w.thetas(16), w.x0, w.obs_times, w.observations(), w.C, w.sigma, 200, 3,
                     block_threads=res["block_threads"], schedule=res["schedule"])
    assert np.array_equal(a["loglik"], b["loglik"])
