"""Exact likelihood of the birth-death network (test infrastructure only).

Network: 0 -> X at rate k1, X -> 0 at rate k2 * x (the paper's first example,
Sec. "The stochastic birth-death Model").  Observations y_k = c x(t_k) + e_k,
e_k ~ N(0, sigma^2).

The paper verifies its sampler against the finite state projection (FSP) of
the chemical master equation (Supp. "posterior verification", RNA model).  For
the birth-death network this is the forward algorithm of a hidden Markov model
on the truncated state space {0..nmax}: transition matrices exp(Q dt) of the
truncated generator, emission N(y; c n, sigma^2).  Probability that leaves the
window (a birth from nmax) goes to an absorbing sink and is dropped, so the
truncated value is a lower bound; ``leak`` reports that mass.

Two independent routes to the transition law are provided:
  * ``transition_expm``: scipy's matrix exponential of the truncated generator;
  * ``transition_closed``: the closed-form law X(t) | X(0)=n ~
    Binomial(n, e^{-k2 t}) (+) Poisson(k1 (1 - e^{-k2 t}) / k2)
    (survivors of the n initial molecules plus an immigration-death
    Poisson part), convolved.
"""
from __future__ import annotations

import numpy as np
from scipy import linalg, stats


def generator(k1: float, k2: float, nmax: int) -> np.ndarray:
    """Generator on {0..nmax} plus a sink state nmax+1 that absorbs births from nmax."""
    n = nmax + 2
    Q = np.zeros((n, n))
    for x in range(nmax + 1):
        Q[x, x + 1] += k1               # birth (from nmax it enters the sink)
        if x > 0:
            Q[x, x - 1] += k2 * x       # death
        Q[x, x] = -(k1 + k2 * x)
    return Q


def transition_expm(k1: float, k2: float, dt: float, nmax: int) -> np.ndarray:
    """P[i, j] = P(X(t+dt) = j | X(t) = i) on the truncated window, i, j <= nmax."""
    P = linalg.expm(generator(k1, k2, nmax) * dt)
    return P[: nmax + 1, : nmax + 1]


def transition_closed(k1: float, k2: float, dt: float, nmax: int) -> np.ndarray:
    """Closed-form transition law (untruncated), restricted to 0..nmax."""
    p = np.exp(-k2 * dt)
    lam = k1 * (1.0 - p) / k2
    m = np.arange(nmax + 1)
    pois = stats.poisson.pmf(m, lam)
    P = np.zeros((nmax + 1, nmax + 1))
    for i in range(nmax + 1):
        b = stats.binom.pmf(np.arange(i + 1), i, p)
        P[i] = np.convolve(b, pois)[: nmax + 1]
    return P


def loglik(k1: float, k2: float, x0: int, obs_times, y, c: float = 1.0, sigma: float = 1.0,
           nmax: int = 200, transition=transition_expm, x0_hi: int | None = None,
           obs_offset: float = 0.0, obs_var: float = 0.0):
    """Exact (truncated) log p(y | k1, k2) of one trajectory, and the leaked mass.

    The forward recursion follows the same factorisation as the paper's filter:
    log p(y) = sum_k log p(y_k | y_{<k}), Supp. I.  Optional model extensions
    (the Lac-Gfp example's forms): the initial count uniform on x0..x0_hi, and
    the emission N(y; obs_offset + c n, sigma^2 + obs_var n).
    """
    obs_times = np.asarray(obs_times, float)
    y = np.asarray(y, float).reshape(-1)
    states = np.arange(nmax + 1)
    alpha = np.zeros(nmax + 1)
    if x0_hi is None:
        alpha[x0] = 1.0
    else:
        alpha[x0:x0_hi + 1] = 1.0 / (x0_hi - x0 + 1)
    sd = np.sqrt(sigma ** 2 + obs_var * states)
    t_prev = 0.0
    L = 0.0
    leak = 0.0
    cache = {}
    for k, t in enumerate(obs_times):
        dt = float(t - t_prev)
        if dt > 0:
            key = round(dt, 12)
            if key not in cache:
                cache[key] = transition(k1, k2, dt, nmax)
            P = cache[key]
            mass_in = alpha.sum()
            alpha = alpha @ P
            leak += mass_in - alpha.sum()
        emis = stats.norm.pdf(y[k], loc=obs_offset + c * states, scale=sd)
        alpha = alpha * emis
        ck = alpha.sum()
        L += np.log(ck)
        alpha = alpha / ck
        t_prev = t
    return L, leak
