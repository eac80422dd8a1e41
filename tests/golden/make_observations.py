"""Write tests/golden/observations.json: the synthetic observed trajectories.

For each workload, T paths of the network are simulated at the data-generating
theta* from x0 with the test oracle's direct-method simulator (data seed of the
workload), and Gaussian measurement noise N(0, sigma_p^2) is added to C x(t_k)
(the observation model of Sec. "General Task": Y_t ~ p(. | X_t, theta)).

Run from the repository root:  python tests/golden/make_observations.py
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
from paper_1606_08281_gb300 import workloads  # noqa: E402


def simulate(w: workloads.Workload) -> dict:
    states, fired, status = pf_oracle.ssa_paths(w.net, w.theta_star, w.x0, w.obs_times, w.T,
                                                seed=w.data_seed)
    assert (status == 0).all()
    noise_rng = np.random.default_rng(w.data_seed + 100)
    y = np.einsum("pu,tku->tkp", w.C, states.astype(np.float64))
    y = y + noise_rng.normal(size=y.shape) * w.sigma[None, None, :]
    return {
        "y": y.tolist(),
        "x_true": states.tolist(),
        "theta_star": w.theta_star.tolist(),
        "x0": w.x0.tolist(),
        "obs_times": w.obs_times.tolist(),
        "events": fired.tolist(),
        "data_seed": w.data_seed,
        "noise_seed": w.data_seed + 100,
    }


def main() -> None:
    out = {}
    for name, make in workloads.WORKLOADS.items():
        w = make()
        out[name] = simulate(w)
        print(name, "events per path:", out[name]["events"][:4], "...")
    with open(workloads.OBSERVATIONS_PATH, "w") as f:
        json.dump(out, f, indent=None, separators=(",", ":"))
        f.write("\n")


if __name__ == "__main__":
    main()
