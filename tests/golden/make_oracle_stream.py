"""Write tests/golden/oracle_stream.json: a fingerprint of the oracle's random
stream and of its filter on fixed small problems.

The oracle's results are a deterministic function of the seed because both
implementations draw the same counter-based Philox words and turn them into
the same variates (Exp(1) by a 2048-layer ziggurat, the selection uniform, the
resampling word, the initial-state words).  This file freezes that definition:
a later change to any of these steps changes the fingerprint, and the test
that reads it (tests/test_oracle_stream_frozen.py) fails until the change is
made deliberately and the file is written again.

Run from the repository root:  python tests/golden/make_oracle_stream.py
Only the oracle and numpy are used; the CUDA library is not involved.
"""
from __future__ import annotations

import json
import sys
from pathlib import Path

import numpy as np

ROOT = Path(__file__).resolve().parents[2]
sys.path.insert(0, str(ROOT))

from oracle import pf_oracle  # noqa: E402
from paper_1606_08281_gb300 import workloads as W  # noqa: E402

OUT = Path(__file__).resolve().parent / "oracle_stream.json"
VARIATE_SEED, N_VARIATES = 20160626, 1 << 16

# (workload, theta rows, trajectories, observation times, particles, seed)
FILTER_CASES = [("birth_death", 8, 1, 20, 64, 1003), ("gene_expression", 4, 2, 8, 50, 2003),
                ("cascade", 2, 2, 4, 40, 3003), ("lac_gfp", 2, 1, 5, 30, 6003)]


def fingerprint() -> dict:
    ev = pf_oracle.exp_variates(VARIATE_SEED, N_VARIATES)
    out = {"variates": {"seed": VARIATE_SEED, "n": N_VARIATES,
                        "first": [float(v).hex() for v in ev[:32]],
                        "sum": float(ev.sum()).hex(),
                        "n_above_5": int((ev > 5.0).sum())},
           "filters": {}}
    for name, M, T, K, N, seed in FILTER_CASES:
        w = W.get(name).subset(T=T, K=K)
        r = pf_oracle.pf_loglik(w.net, w.thetas(M), w.x0, w.obs_times, w.observations(), w.C,
                                w.sigma, N, seed, model=w.model)
        out["filters"][name] = {"M": M, "T": T, "K": K, "N": N, "seed": seed,
                                "events": r["events"].astype(int).tolist(),
                                "digest": [[f"{int(d):016x}" for d in row] for row in r["digest"]],
                                "status": r["status"].astype(int).tolist(),
                                "ll_traj": [[float(v).hex() for v in row] for row in r["ll_traj"]]}
    return out


if __name__ == "__main__":
    OUT.write_text(json.dumps(fingerprint(), indent=1) + "\n")
    print(OUT)
