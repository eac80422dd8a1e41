"""World-size-2 gloo test of the multi-rank bookkeeping on CPU: per-rank theta
batches, row sharding, max-over-ranks timing and gathering a sharded batch.
The filters themselves need no exchange (each rank runs whole filters); here
the oracle stands in for the per-rank compute so the test runs without a GPU."""
from __future__ import annotations

import os
import socket

import numpy as np
import torch.multiprocessing as mp

from paper_1606_08281_gb300 import multi
from paper_1606_08281_gb300 import workloads as W


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from oracle import pf_oracle
    w = W.birth_death()
    th = w.thetas(10)
    sl = multi.shard_rows(len(th), rank, world)
    r = pf_oracle.pf_loglik(w.net, th[sl], w.x0, w.obs_times, w.observations(), w.C, w.sigma, 20,
                            w.filter_seed, theta_ids=np.arange(sl.start, sl.stop))
    full = multi.gather_rows(r["loglik"], len(th))
    t = multi.max_over_ranks(0.5 + rank)
    own = multi.rank_thetas(w, rank)
    out[rank] = (full, t, own[:3].copy())
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_gloo_sharding_and_timing():
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    from oracle import pf_oracle
    w = W.birth_death()
    th = w.thetas(10)
    ref = pf_oracle.pf_loglik(w.net, th, w.x0, w.obs_times, w.observations(), w.C, w.sigma, 20,
                              w.filter_seed)["loglik"]
    for rank in range(world):
        full, t, own = out[rank]
        assert np.array_equal(full, ref)          # sharded == unsharded, row order kept
        assert t == 1.5                           # max over ranks
    assert np.array_equal(out[0][2], w.thetas(3))
    assert not np.array_equal(out[0][2], out[1][2])   # independent batches per rank


def test_shard_rows_cover_exactly():
    for M in (0, 1, 7, 4096):
        for world in (1, 2, 3, 8):
            rows = np.concatenate([np.arange(M)[multi.shard_rows(M, r, world)] for r in range(world)])
            assert np.array_equal(rows, np.arange(M))
