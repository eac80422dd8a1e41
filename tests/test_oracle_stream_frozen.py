"""The oracle's random stream is frozen (CPU).

tests/golden/oracle_stream.json, written by tests/golden/make_oracle_stream.py
from the oracle alone, fingerprints the Exp(1) variates of a fixed draw
sequence and the complete histories (events, digests) of small filters on
every workload.  Integers must match exactly; floating-point values may differ
by a few units in the last place (another host C library's exp/log), which no
change to the stream's definition could stay within.
"""
from __future__ import annotations

import json
from pathlib import Path

import numpy as np

GOLDEN = Path(__file__).resolve().parent / "golden" / "oracle_stream.json"


def test_oracle_stream_matches_its_frozen_fingerprint():
    import sys
    sys.path.insert(0, str(GOLDEN.parent))
    import make_oracle_stream as mk
    want = json.loads(GOLDEN.read_text())
    got = mk.fingerprint()
    a, b = want["variates"], got["variates"]
    assert (a["seed"], a["n"], a["n_above_5"]) == (b["seed"], b["n"], b["n_above_5"])
    fa = np.array([float.fromhex(v) for v in a["first"]])
    fb = np.array([float.fromhex(v) for v in b["first"]])
    np.testing.assert_array_max_ulp(fa, fb, maxulp=4)
    assert abs(float.fromhex(a["sum"]) - float.fromhex(b["sum"])) <= 1e-9 * float.fromhex(a["sum"])
    assert set(want["filters"]) == set(got["filters"])
    for name, fw in want["filters"].items():
        fg = got["filters"][name]
        for k in ("M", "T", "K", "N", "seed", "events", "digest", "status"):
            assert fw[k] == fg[k], (name, k)
        la = np.array([[float.fromhex(v) for v in row] for row in fw["ll_traj"]])
        lb = np.array([[float.fromhex(v) for v in row] for row in fg["ll_traj"]])
        np.testing.assert_allclose(lb, la, rtol=1e-12, atol=0)
