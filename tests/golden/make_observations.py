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
    if w.model is not None:
        return simulate_model(w)
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


def simulate_model(w: workloads.Workload) -> dict:
    """Workloads with the Lac-Gfp extensions: each trajectory starts from its
    own draw of the uniform initial distribution, rates are composed, and the
    observation is y = offset + C x + sqrt(sigma^2 + V x) * N(0, 1)."""
    md = w.model
    x0_rng = np.random.default_rng(w.data_seed + 200)
    noise_rng = np.random.default_rng(w.data_seed + 100)
    lo, hi = w.x0, np.asarray(md["x0_hi"], np.int32)
    all_states, all_fired, x0s = [], [], []
    for traj in range(w.T):
        x0 = x0_rng.integers(lo, hi + 1).astype(np.int32)
        states, fired, status = pf_oracle.ssa_paths(w.net, w.theta_star, x0, w.obs_times, 1,
                                                    seed=w.data_seed + traj,
                                                    rate_coef=md["rate_coef"])
        assert (status == 0).all()
        all_states.append(states[0])
        all_fired.append(int(fired[0]))
        x0s.append(x0.tolist())
    states = np.array(all_states)                                   # [T][K][U]
    xs = states.astype(np.float64)
    mean = np.asarray(md["obs_offset"])[None, None, :] + np.einsum("pu,tku->tkp", w.C, xs)
    var = (w.sigma ** 2)[None, None, :] + np.einsum("pu,tku->tkp", np.asarray(md["obs_var"]), xs)
    y = mean + noise_rng.normal(size=mean.shape) * np.sqrt(var)
    return {
        "y": y.tolist(),
        "x_true": states.tolist(),
        "theta_star": w.theta_star.tolist(),
        "x0": x0s,
        "obs_times": w.obs_times.tolist(),
        "events": all_fired,
        "data_seed": w.data_seed,
        "noise_seed": w.data_seed + 100,
        "x0_seed": w.data_seed + 200,
    }


def simulate_erk(w) -> dict:
    """The Erk ODE model at theta_bar for each input pattern, plus
    N(0, sigma^2) measurement noise (sigma = theta_bar[32])."""
    from oracle import ode
    mean = ode.observe(w.theta_bar, w.patterns, w.obs_times)
    rng = np.random.default_rng(w.data_seed)
    y = mean + rng.normal(size=mean.shape) * w.theta_bar[32]
    return {"y": y.tolist(), "mean": mean.tolist(), "theta_bar": w.theta_bar.tolist(),
            "obs_times": w.obs_times.tolist(), "data_seed": w.data_seed}


def main() -> None:
    out = {}
    for name, make in workloads.WORKLOADS.items():
        w = make()
        out[name] = simulate(w)
        print(name, "events per path:", out[name]["events"][:4], "...")
    out["erk"] = simulate_erk(workloads.erk())
    print("erk: FRET range", min(map(min, out["erk"]["y"])), max(map(max, out["erk"]["y"])))
    with open(workloads.OBSERVATIONS_PATH, "w") as f:
        json.dump(out, f, indent=None, separators=(",", ":"))
        f.write("\n")


if __name__ == "__main__":
    main()
