"""Pins of the ODE oracle (oracle/ode.py) for the Egf-Ras-Raf-Mek-Erk model,
against which the CUDA ODE likelihood is compared.

Each pin reduces a part of the model to mathematics that does not go through
the oracle's own formula: the six active/inactive pairs are conserved; the
receptor pair under a constant input and the dusp/DUSP chain without active
ERK have closed-form solutions; the Ras layer settles at the root of its
Michaelis-Menten balance; the FRET ratio has closed forms at no and at full
ERK activation; a noise-free trajectory scores the Gaussian normaliser alone.
Planted mistakes in a copy of ode.py must each fail a pin.
"""
from __future__ import annotations

import inspect
import types

import numpy as np
import pytest
from scipy import optimize

from oracle import ode
from paper_1606_08281_gb300 import workloads as W

PAIRS = [(0, 1), (2, 3), (4, 5), (6, 7), (8, 9), (10, 11)]


def check_conservation(o):
    w = W.erk()
    for th in [w.theta_bar, *w.thetas(3)]:
        for st, sv in w.patterns[:3]:
            X = o.solve(th, st, sv, w.obs_times)
            x0 = o.initial_state(th)
            for a, b in PAIRS:
                assert np.allclose(X[:, a] + X[:, b], x0[a] + x0[b], rtol=1e-9, atol=1e-13), (a, b)


def test_active_inactive_pairs_conserved():
    check_conservation(ode)


def check_receptor_closed_form(o):
    """EGFR* under a constant input u from t = 0, EGFR*(0) = 0:
    EGFR*(t) = E0 k1 u / (k1 u + g1) (1 - exp(-(k1 u + g1) t))."""
    th = W.ERK_THETA_BAR.copy()
    th[0], th[1], th[27] = 0.3, 0.05, 0.8
    u = 2.0
    t = 2.0 * np.arange(1, 61)
    X = o.solve(th, [0.0], [u], t)
    s = th[0] * u + th[1]
    want = th[27] * th[0] * u / s * (1.0 - np.exp(-s * t))
    assert np.allclose(X[:, 1], want, rtol=1e-9, atol=1e-13)


def test_receptor_closed_form():
    check_receptor_closed_form(ode)


def check_dusp_closed_form(o):
    """With k5 = 0 ERK* stays 0, so dusp relaxes to dusp_basal at rate
    a = log10(2)/90 and DUSP follows the resonant chain:
    dusp = b + (d0 - b) e^{-at},  DUSP = b + (d0 - b)(1 + a t) e^{-at}."""
    th = W.ERK_THETA_BAR.copy()
    th[15] = 0.0
    th[24], th[29] = 0.05, 0.4
    t = 2.0 * np.arange(1, 61)
    X = o.solve(th, [0.0], [1.0], t)
    a, b, d0 = np.log10(2.0) / 90.0, th[24], th[29]
    assert np.allclose(X[:, 9], 0.0, atol=1e-15)
    assert np.allclose(X[:, 12], b + (d0 - b) * np.exp(-a * t), rtol=1e-9)
    assert np.allclose(X[:, 13], b + (d0 - b) * (1.0 + a * t) * np.exp(-a * t), rtol=1e-9)


def test_dusp_closed_form():
    check_dusp_closed_form(ode)


def check_ras_steady_state(o):
    """Constant input, fast layers: EGFR* -> E0 k1 u/(k1 u + g1) and Ras* settles
    at the root R of k2 EGFR* (Rt - R)/(K2 + Rt - R) = g2 R/(D2 + R)."""
    th = W.ERK_THETA_BAR.copy()
    th[0], th[1], th[2], th[3], th[4], th[5], th[27] = 5.0, 1.0, 5.0, 0.3, 2.0, 0.2, 0.9
    X = o.solve(th, [0.0], [1.0], [60.0, 120.0])
    Ea = th[27] * th[0] / (th[0] + th[1])
    Rt = 0.1
    f = lambda R: th[2] * Ea * (Rt - R) / (th[3] + Rt - R) - th[4] * R / (th[5] + R)  # noqa: E731
    R = optimize.brentq(f, 0.0, Rt, xtol=1e-15)
    assert np.isclose(X[-1, 3], R, rtol=1e-8)


def test_ras_steady_state():
    check_ras_steady_state(ode)


def check_fret_limits(o):
    th = W.ERK_THETA_BAR.copy()
    th[30], th[31], th[33], th[34], th[35] = 0.4, 2.0, 0.3, 1.5, 0.7
    x = o.initial_state(th)                       # ERK* = 0
    assert np.isclose(o.fret(x, th), th[31] * th[30], rtol=1e-15)
    x[8], x[9] = 0.0, 0.2                         # all ERK active
    want = th[31] * (th[33] * th[34] / ((1.0 - th[33]) * th[35]) + th[30])
    assert np.isclose(o.fret(x, th), want, rtol=1e-14)


def test_fret_limits():
    check_fret_limits(ode)


def check_noise_free_loglik(o):
    """y equal to the mean trajectory: the log-likelihood is the Gaussian
    normaliser, -n (log sigma + log(2 pi) / 2)."""
    w = W.erk()
    th = w.theta_bar
    y = o.observe(th, w.patterns, w.obs_times)
    L, per = o.loglik(th, w.patterns, w.obs_times, y)
    n = y.size
    assert np.isclose(L, -n * (np.log(th[32]) + 0.5 * np.log(2 * np.pi)), rtol=1e-12)


def test_noise_free_loglik():
    check_noise_free_loglik(ode)


MUTANTS = {
    "pair_mixed": ("-v4, v4, -v5", "-v4, v3, -v5", check_conservation),
    "dusp_decay_rate": ("- dusp * a\n", "- dusp * 2.0 * a\n", check_dusp_closed_form),
    "DUSP_no_decay": ("dDUSP = dusp * a - DUSP * a", "dDUSP = dusp * a", check_dusp_closed_form),
    "receptor_swapped": ("v1 = k1 * egf * EGFR - g1 * EGFRa", "v1 = k1 * egf * EGFRa - g1 * EGFR",
                         check_receptor_closed_form),
    "ras_michaelis_argument": ("k2 * EGFRa * Ras / (K2 + Ras)", "k2 * EGFRa * Ras / (K2 + Rasa)",
                               check_ras_steady_state),
    "fret_efficiency": ("(ERK + (1.0 - E) * ERKa)", "(ERK + E * ERKa)", check_fret_limits),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_ode_pin_detects_mutant(name):
    old, new, check = MUTANTS[name]
    src = inspect.getsource(ode)
    assert src.count(old) == 1, old
    mod = types.ModuleType("ode_variant")
    exec(compile(src.replace(old, new), "ode_variant", "exec"), mod.__dict__)
    mod.solve.__defaults__ = mod.solve.__defaults__[:-1] + (200_000,)   # a diverging mutant ends fast
    with pytest.raises((AssertionError, ValueError, RuntimeError)):
        check(mod)
