"""bench.py's reference arm (the oracle on the host cores) prints one JSON line
with the contract's keys and the same metric, unit and workload config as the
GPU arm (CPU only: the small birth-death workload, about 20 s)."""
from __future__ import annotations

import json
import subprocess
import sys
from pathlib import Path

ROOT = Path(__file__).resolve().parents[1]


def test_reference_arm_line():
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload",
                          "birth_death", "--steps", "1", "--warmup", "0"], cwd=ROOT,
                         capture_output=True, text=True, timeout=300, check=True).stdout
    lines = [ln for ln in out.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, out
    line = json.loads(lines[0])
    sys.path.insert(0, str(ROOT))
    import bench
    from paper_1606_08281_gb300 import workloads as W
    assert line["impl"] == "reference"
    assert line["metric"] == "theta-likelihoods/s" and line["unit"] == "theta-likelihoods/s"
    assert line["higher_is_better"] is True and line["steps"] == 1 and line["warmup"] == 0
    assert line["config"] == bench.config_of(W.get("birth_death"))
    assert line["value"] > 0 and line["ms_per_step"] > 0
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"] and cb["value"] == line["value"]
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["unit"] == line["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_exact_oracle_legs():
    """The FSP and ODE oracle legs of `bench.py --mode fsp / ode` count rows
    finished in a short window (a few seconds of host work each)."""
    sys.path.insert(0, str(ROOT))
    import bench
    for leg, name, M in [("fsp", "telegraph", 64), ("ode", "erk", 64)]:
        r = bench.exact_baseline(leg, name, M, 3.0)
        assert r["kind"] == "oracle" and r["cores"] >= 1 and r["unit"] == "theta-likelihoods/s"
        assert r["value"] > 0 and r["wall_s"] <= 10.0, r
        assert f"{M}-row {name} batch" in r["sample"]


def test_reference_arm_of_the_ode_mode():
    """--mode ode --impl reference times the ODE oracle on the GPU arm's batch
    and config (64 rows: a few seconds)."""
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--mode", "ode",
                          "--ode-theta", "64", "--steps", "1", "--warmup", "0"], cwd=ROOT,
                         capture_output=True, text=True, timeout=300, check=True).stdout
    line = json.loads([ln for ln in out.splitlines() if ln.startswith("{")][-1])
    sys.path.insert(0, str(ROOT))
    import bench
    assert line["impl"] == "reference" and line["mode"] == "ode"
    assert line["metric"] == "ODE theta-likelihoods/s" and line["higher_is_better"] is True
    assert line["config"] == bench.ode_config(bench.ode_workload(64))
    assert line["value"] > 0 and line["cpu_baseline"]["kind"] == "oracle"
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
