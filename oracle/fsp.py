"""Exact (truncated) trajectory likelihood by the finite state projection
(test infrastructure only).

The paper obtains the "(almost) exact" likelihood of its RNA model with the
finite state projection of the chemical master equation (Supp. "Verification
of approximated posterior", citing Munsky & Khammash's FSP).  On the box
B = {x : 0 <= x_u <= n_u} the master equation's generator Q moves probability
out of every state x at rate a_0(x) = sum_r a_r(x) and into x + nu_r at rate
a_r(x) when that state lies in B; probability whose next state leaves B is
dropped, so the truncated likelihood is a lower bound and the dropped mass is
reported as the leak.

The observation model is the particle filter's (Supp. I): y_k ~ N(C x, diag
sigma^2), or with the model extensions (mean offset, variance
sigma^2 + V x).  The likelihood factorises over observation times exactly as
the filter's estimate does, log p(y) = sum_k log p(y_k | y_<k), and the
forward algorithm computes each factor:
    alpha <- alpha exp(Q dt_k)            (scipy.sparse.linalg.expm_multiply)
    alpha <- alpha * p(y_k | x);  c_k = sum(alpha);  log p(y) += log c_k
    alpha <- alpha / c_k
States are indexed with the last species fastest:
index(x) = sum_u x_u * stride_u, stride_{U-1} = 1, stride_u = stride_{u+1} (n_{u+1} + 1).
"""
from __future__ import annotations

import numpy as np
from scipy import sparse, stats
from scipy.sparse import linalg as splinalg


def box_states(box_max) -> np.ndarray:
    """All states of the box, [S][U] int64, in index order."""
    box_max = np.asarray(box_max, np.int64)
    grids = np.meshgrid(*[np.arange(n + 1) for n in box_max], indexing="ij")
    return np.stack([g.reshape(-1) for g in grids], axis=1)


def strides(box_max) -> np.ndarray:
    box_max = np.asarray(box_max, np.int64)
    U = len(box_max)
    st = np.ones(U, np.int64)
    for u in range(U - 2, -1, -1):
        st[u] = st[u + 1] * (box_max[u + 1] + 1)
    return st


def reaction_rates(net: dict, theta, model: dict | None = None) -> np.ndarray:
    """theta[rate_index[r]] (or theta[r]), or the composed sums rate_coef @ theta."""
    theta = np.asarray(theta, float)
    R = np.asarray(net["reactants"]).shape[0]
    if model is not None and model.get("rate_coef") is not None:
        return np.asarray(model["rate_coef"], float).reshape(R, len(theta)) @ theta
    ri = net.get("rate_index")
    return theta[np.asarray(ri)] if ri is not None else theta[:R]


def propensities(net: dict, rate, X) -> np.ndarray:
    """Mass-action propensities a_r(x) = rate_r prod_u binom(x_u, p_ru), [S][R]."""
    reac = np.asarray(net["reactants"], np.int64)
    X = np.asarray(X, np.int64)
    h = np.ones((X.shape[0], reac.shape[0]), np.int64)
    for r in range(reac.shape[0]):
        for u in range(reac.shape[1]):
            p = reac[r, u]
            if p == 1:
                h[:, r] *= X[:, u]
            elif p == 2:
                h[:, r] *= X[:, u] * (X[:, u] - 1) // 2
    return h.astype(float) * np.asarray(rate, float)[None, :]


def generator(net: dict, rate, box_max) -> sparse.csr_matrix:
    """Q[i, j] = rate of the jump i -> j inside the box; Q[i, i] = -a_0(x_i)."""
    X = box_states(box_max)
    S = X.shape[0]
    A = propensities(net, rate, X)
    nu = np.asarray(net["products"], np.int64) - np.asarray(net["reactants"], np.int64)
    st = strides(box_max)
    box = np.asarray(box_max, np.int64)
    rows, cols, vals = [], [], []
    for r in range(nu.shape[0]):
        Y = X + nu[r][None, :]
        inside = np.all((Y >= 0) & (Y <= box[None, :]), axis=1) & (A[:, r] > 0)
        rows.append(np.nonzero(inside)[0])
        cols.append(Y[inside] @ st)
        vals.append(A[inside, r])
    rows.append(np.arange(S))
    cols.append(np.arange(S))
    vals.append(-A.sum(axis=1))
    return sparse.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                             shape=(S, S))


def initial(x0, box_max, x0_hi=None) -> np.ndarray:
    """Point mass at x0, or independent uniform integers x0_u..x0_hi_u per species."""
    X = box_states(box_max)
    lo = np.asarray(x0, np.int64)
    hi = lo if x0_hi is None else np.asarray(x0_hi, np.int64)
    inside = np.all((X >= lo[None, :]) & (X <= hi[None, :]), axis=1)
    alpha = inside.astype(float)
    return alpha / alpha.sum()


def log_emission(yk, X, C, sigma, model: dict | None = None) -> np.ndarray:
    """log p(y_k | x) for every state: Gaussian, mean offset + C x, variance
    sigma^2 (+ V x with the model's obs_var)."""
    X = np.asarray(X, float)
    C = np.asarray(C, float)
    P = C.shape[0]
    sigma = np.asarray(sigma, float).reshape(P)
    md = model or {}
    off = np.zeros(P) if md.get("obs_offset") is None else np.asarray(md["obs_offset"], float)
    mean = off[None, :] + X @ C.T
    var = np.broadcast_to(sigma ** 2, mean.shape).copy()
    if md.get("obs_var") is not None:
        var = var + X @ np.asarray(md["obs_var"], float).reshape(P, -1).T
    return stats.norm.logpdf(np.asarray(yk, float)[None, :], mean, np.sqrt(var)).sum(axis=1)


def propagate(Q: sparse.csr_matrix, alpha: np.ndarray, dt: float) -> np.ndarray:
    """alpha exp(Q dt) for a row vector alpha."""
    if dt <= 0:
        return alpha.copy()
    return splinalg.expm_multiply(Q.T.tocsc() * dt, alpha)


def loglik(net: dict, theta, x0, box_max, obs_times, y_traj, C, sigma, model: dict | None = None):
    """FSP log p(y_traj | theta) of one trajectory ([K][P]) and the dropped mass."""
    md = model or {}
    rate = reaction_rates(net, theta, md)
    Q = generator(net, rate, box_max)
    X = box_states(box_max)
    alpha = initial(x0, box_max, md.get("x0_hi"))
    y_traj = np.asarray(y_traj, float).reshape(len(obs_times), -1)
    t_prev, L, leak = 0.0, 0.0, 0.0
    for k, t in enumerate(np.asarray(obs_times, float)):
        mass_in = alpha.sum()
        alpha = propagate(Q, alpha, float(t - t_prev))
        alpha = np.maximum(alpha, 0.0)                 # expm_multiply rounding near zero
        leak += mass_in - alpha.sum()
        le = log_emission(y_traj[k], X, C, sigma, md)
        m = le[alpha > 0].max() if (alpha > 0).any() else le.max()   # shift on the support
        w = alpha * np.exp(le - m)
        c = w.sum()
        L += m + np.log(c)
        alpha = w / c
        t_prev = float(t)
    return float(L), float(leak)


def loglik_batch(net: dict, thetas, x0, box_max, obs_times, y, C, sigma, model: dict | None = None):
    """Per-theta sums over trajectories (y [T][K][P]) and per-(theta, trajectory) values/leaks."""
    thetas = np.atleast_2d(np.asarray(thetas, float))
    y = np.asarray(y, float)
    M, T = thetas.shape[0], y.shape[0]
    ll = np.zeros((M, T))
    leak = np.zeros((M, T))
    for m in range(M):
        for t in range(T):
            ll[m, t], leak[m, t] = loglik(net, thetas[m], x0, box_max, obs_times, y[t], C, sigma,
                                          model)
    return ll.sum(axis=1), ll, leak
