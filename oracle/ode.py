"""Deterministic (ODE) likelihood of the Egf-Ras-Raf-Mek-Erk model
(test infrastructure only).

The paper's third example (Supp. "Egf-Ras-Raf-Mek-Erk model", its reaction
equations and FRET noise model): in a deterministic model the likelihood
needs no particle filter -- solve the ODE for the parameter vector and score
the resulting trajectory under the observation model (Sec. "A realistic
example").  The state is the 14 concentrations
    EGFR, EGFR*, Ras, Ras*, Raf, Raf*, MEK, MEK*, ERK, ERK*, NFB, NFB*, dusp, DUSP
and the observation of each input pattern at each time is the FRET ratio
    R(t) = lam (ERK* E f_AA / ((ERK + (1 - E) ERK*) f_DD) + bg) + N(0, sigma^2).

theta (36 entries, the paper's unknowns, in this order):
    0 k1, 1 gamma1, 2 k2, 3 K2, 4 gamma2, 5 D2, 6 k3, 7 K3, 8 K_NFB, 9 gamma3,
    10 D3, 11 k4, 12 K4, 13 gamma4, 14 D4, 15 k5, 16 K5, 17 gamma5, 18 D5,
    19 k6, 20 K6, 21 K6R, 22 gamma6, 23 D6, 24 dusp_basal, 25 dusp_ind,
    26 K_dusp, 27 EGFR(0), 28 NFB(0), 29 dusp(0) = DUSP(0),
    30 bg, 31 lam, 32 sigma, 33 E, 34 f_AA, 35 f_DD.
Fixed: T_dusp = T_DUSP = 90 min; Ras(0) = 0.1, Raf(0) = 0.7, MEK(0) = 0.68,
ERK(0) = 0.26, active forms 0.  The dusp equations carry log10(2) / T as
printed in the paper.  egf_input(t) is piecewise constant (value v_i from
switch time s_i on); the solution is integrated piece by piece between
switch times with scipy's 8th-order Dormand-Prince integrator (a library
routine) at rtol 1e-11, observation times from its dense output.
"""
from __future__ import annotations

import numpy as np
from scipy import integrate, stats

N_STATE = 14
N_THETA = 36
T_HALF = 90.0
FIXED_INIT = {2: 0.1, 4: 0.7, 6: 0.68, 8: 0.26}
NAMES = ["k1", "gamma1", "k2", "K2", "gamma2", "D2", "k3", "K3", "K_NFB", "gamma3", "D3", "k4",
         "K4", "gamma4", "D4", "k5", "K5", "gamma5", "D5", "k6", "K6", "K6R", "gamma6", "D6",
         "dusp_basal", "dusp_ind", "K_dusp", "EGFR0", "NFB0", "dusp0", "bg", "lam", "sigma", "E",
         "f_AA", "f_DD"]


def initial_state(theta) -> np.ndarray:
    x = np.zeros(N_STATE)
    for i, v in FIXED_INIT.items():
        x[i] = v
    x[0] = theta[27]
    x[10] = theta[28]
    x[12] = x[13] = theta[29]
    return x


def rhs(x, theta, egf: float) -> np.ndarray:
    """The reaction equations of the model (Supp. "Reaction Equations")."""
    (k1, g1, k2, K2, g2, D2, k3, K3, KNFB, g3, D3, k4, K4, g4, D4, k5, K5, g5, D5, k6, K6, K6R,
     g6, D6, dbas, dind, Kd) = theta[:27]
    EGFR, EGFRa, Ras, Rasa, Raf, Rafa, MEK, MEKa, ERK, ERKa, NFB, NFBa, dusp, DUSP = x
    v1 = k1 * egf * EGFR - g1 * EGFRa
    v2 = k2 * EGFRa * Ras / (K2 + Ras) - g2 * Rasa / (D2 + Rasa)
    v3 = (k3 * Rasa * Raf / (K3 + Raf) * KNFB ** 2 / (KNFB ** 2 + NFBa ** 2)
          - g3 * Rafa / (D3 + Rafa))
    v4 = k4 * Rafa * MEK / (K4 + MEK) - g4 * MEKa / (D4 + MEKa)
    v5 = k5 * MEKa * ERK / (K5 + ERK) - g5 * DUSP * ERKa / (D5 + ERKa)
    v6 = (k6 * ERKa * NFB / (K6 + NFB) * EGFRa ** 2 / (K6R ** 2 + EGFRa ** 2)
          - g6 * NFBa / (D6 + NFBa))
    a = np.log10(2.0) / T_HALF
    ddusp = dbas * (1.0 + dind * ERKa ** 2 / (Kd + ERKa ** 2)) * a - dusp * a
    dDUSP = dusp * a - DUSP * a
    return np.array([-v1, v1, -v2, v2, -v3, v3, -v4, v4, -v5, v5, -v6, v6, ddusp, dDUSP])


def fret(x, theta) -> float:
    """Mean FRET ratio of a state (Supp. "Noise Model")."""
    bg, lam, E, fAA, fDD = theta[30], theta[31], theta[33], theta[34], theta[35]
    ERK, ERKa = x[8], x[9]
    return lam * (ERKa * E * fAA / ((ERK + (1.0 - E) * ERKa) * fDD) + bg)


class BudgetError(RuntimeError):
    """The integration needed more right-hand-side evaluations than allowed."""


def solve(theta, switch_times, switch_values, obs_times, rtol=1e-11, atol=1e-14,
          method="DOP853", max_rhs: int = 2_000_000) -> np.ndarray:
    """States at the observation times, [K][14]: integrated from 0 piece by
    piece between consecutive input switch times (the right-hand side is
    smooth inside a piece), observation times read from the integrator's
    dense output.  More than max_rhs right-hand-side evaluations in total
    (a stiff or diverging solution) raise BudgetError."""
    theta = np.asarray(theta, float)
    st = np.asarray(switch_times, float)
    sv = np.asarray(switch_values, float)
    obs = np.asarray(obs_times, float)
    ends = np.unique(np.concatenate([st[st > 0.0], [obs[-1]]]))
    ends = ends[ends <= obs[-1]]
    x = initial_state(theta)
    out = np.zeros((len(obs), N_STATE))
    t = 0.0
    calls = [0]

    def f(_t, z, egf):
        calls[0] += 1
        if calls[0] > max_rhs:
            raise BudgetError(f"more than {max_rhs} right-hand-side evaluations")
        return rhs(z, theta, egf)

    for t1 in ends:
        idx = np.searchsorted(st, t, side="right") - 1     # input in force on [t, t1)
        egf = sv[idx] if idx >= 0 else 0.0
        inside = (obs > t) & (obs <= t1)
        t_eval = np.unique(np.concatenate([obs[inside], [t1]]))      # ends with t1
        sol = integrate.solve_ivp(f, (t, t1), x, method=method, rtol=rtol, atol=atol,
                                  t_eval=t_eval, args=(egf,))
        if not sol.success:
            raise RuntimeError(sol.message)
        if inside.any():
            out[inside] = sol.y.T[np.searchsorted(t_eval, obs[inside])]
        x = sol.y[:, -1]
        t = t1
    return out


def loglik(theta, patterns, obs_times, y):
    """Sum over input patterns of sum_k log N(y[p][k]; R(x(t_k)), sigma^2);
    patterns = [(switch_times, switch_values), ...], y [n_patterns][K].
    Returns (total, per-pattern values)."""
    theta = np.asarray(theta, float)
    per = []
    for p, (st, sv) in enumerate(patterns):
        X = solve(theta, st, sv, obs_times)
        R = np.array([fret(x, theta) for x in X])
        per.append(float(stats.norm.logpdf(np.asarray(y[p], float), R, theta[32]).sum()))
    return float(np.sum(per)), np.array(per)


def observe(theta, patterns, obs_times):
    """Mean FRET trajectories [n_patterns][K] (for synthesising data)."""
    return np.array([[fret(x, theta) for x in solve(theta, st, sv, obs_times)]
                     for st, sv in patterns])
