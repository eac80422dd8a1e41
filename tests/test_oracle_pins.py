"""Pins of the oracle to facts outside itself (CPU only).

Each test checks the oracle against something the paper or mathematics fixes:
published known-answer vectors, closed-form laws of simple networks, exact
likelihoods from the forward algorithm, special cases with closed forms, and
the defining properties of systematic resampling.  The mutation tests in
test_oracle_mutants.py show that plausible mistakes in the oracle fail them.
"""
from __future__ import annotations

import numpy as np
import pytest
from scipy import stats

from oracle import exact_bd
from oracle import pf_oracle
from paper_1606_08281_gb300 import workloads as W

BD = W.birth_death_network()
GE = W.gene_expression_network()
DIMER = {"reactants": np.array([[2]], np.int32), "products": np.array([[0]], np.int32),
         "rate_index": None}
HETERO = {"reactants": np.array([[1, 1, 0]], np.int32), "products": np.array([[0, 0, 1]], np.int32),
          "rate_index": None}
REVERSIBLE = {"reactants": np.array([[1, 1, 0], [0, 0, 1]], np.int32),
              "products": np.array([[0, 0, 1], [1, 1, 0]], np.int32), "rate_index": None}


def orc():
    return pf_oracle.default()


# ---------------------------------------------------------------- Philox ---
def check_philox(o, kat_vectors):
    for ctr, key, want in kat_vectors:
        got = o.philox4x32_10(ctr, key)
        assert [int(v) for v in got] == want


def test_philox_known_answers(kat_vectors):
    """Philox4x32-10 reproduces the Random123 known-answer vectors (Salmon et al. SC'11)."""
    check_philox(orc(), kat_vectors)


# ------------------------------------------------- exponential variates ---
def check_exp_variates(o, n=400_000):
    """The ziggurat generator's law is Exp(1): Kolmogorov-Smirnov against the
    exponential CDF, mean and variance 1, and the tail beyond the ziggurat's
    base x = r = 10.023 (handled by a separate branch) has mass exp(-r)."""
    e = o.exp_variates(2024, n)
    assert (e >= 0).all()
    assert stats.kstest(e, "expon").pvalue > 1e-3
    assert abs(e.mean() - 1.0) < 5 / np.sqrt(n)
    assert abs(e.var() - 1.0) < 5 * np.sqrt(8.0 / n)
    r = 10.02289706840504086041
    big = o.exp_variates(77, 4_000_000)
    k = int((big > r).sum())
    lam = 4_000_000 * np.exp(-r)
    assert abs(k - lam) < 5 * np.sqrt(lam)
    # just below the base strip and inside the wedges the density is exp(-x) too
    for a, b in [(0.0, 0.01), (2.0, 2.5), (5.0, 10.0)]:
        want = np.exp(-a) - np.exp(-b)
        got = np.mean((big >= a) & (big < b))
        assert abs(got - want) < 5 * np.sqrt(want / 4_000_000)


def test_exponential_variates_law():
    check_exp_variates(orc())


# ------------------------------------------------------- exact likelihood ---
@pytest.mark.parametrize("k1,k2,dt", [(10.0, 0.2, 1.0), (30.0, 0.9, 0.5), (3.0, 0.05, 2.0)])
def test_exact_transition_two_routes(k1, k2, dt):
    """expm of the truncated generator equals the closed-form Binomial (+) Poisson law."""
    A = exact_bd.transition_expm(k1, k2, dt, 200)
    B = exact_bd.transition_closed(k1, k2, dt, 200)
    rows = slice(0, 120)                                  # far from the truncation edge
    assert np.max(np.abs(A[rows] - B[rows])) < 1e-12
    assert np.allclose(B.sum(axis=1)[rows], 1.0, atol=1e-12)


def test_exact_loglik_two_routes():
    w = W.birth_death()
    y = w.observations()[0, :, 0]
    for k1, k2 in [(10.0, 0.2), (20.0, 0.5), (4.0, 0.1)]:
        La, leak = exact_bd.loglik(k1, k2, 10, w.obs_times, y, 1.0, 1.0, 200)
        Lb, _ = exact_bd.loglik(k1, k2, 10, w.obs_times, y, 1.0, 1.0, 200,
                                transition=exact_bd.transition_closed)
        assert abs(leak) < 1e-12
        assert abs(La - Lb) < 1e-9


# --------------------------------------------------------- simulator law ---
def chi2_pvalue(samples, pmf):
    """Pearson chi-square p-value, bins merged until each expects >= 5."""
    n = len(samples)
    counts = np.bincount(samples, minlength=len(pmf))[: len(pmf)].astype(float)
    counts[-1] += np.sum(samples >= len(pmf))
    exp_ = pmf * n
    exp_[-1] += max(0.0, n - exp_.sum())
    obs_b, exp_b, acc_o, acc_e = [], [], 0.0, 0.0
    for o, e in zip(counts, exp_):
        acc_o += o
        acc_e += e
        if acc_e >= 5:
            obs_b.append(acc_o)
            exp_b.append(acc_e)
            acc_o = acc_e = 0.0
    if acc_e > 0 and obs_b:
        obs_b[-1] += acc_o
        exp_b[-1] += acc_e
    chi2 = np.sum((np.array(obs_b) - np.array(exp_b)) ** 2 / np.array(exp_b))
    return stats.chi2.sf(chi2, len(obs_b) - 1)


def check_birth_death_law(o, n=20000):
    k1, k2, x0 = 10.0, 0.2, 10
    times = np.array([0.5, 2.0, 10.0])
    states, _, status = o.ssa_paths(BD, [k1, k2], [x0], times, n, seed=77)
    assert (status == 0).all()
    assert (states >= 0).all()                      # molecule counts never go negative
    t_prev = 0.0
    for k, t in enumerate(times):
        pmf = exact_bd.transition_closed(k1, k2, t, 200)[x0]
        assert chi2_pvalue(states[:, k, 0], pmf) > 1e-3, f"t={t}"
        t_prev = t
    return t_prev


def test_ssa_birth_death_transient_law():
    """X(t)|X(0)=10 ~ Binomial(10, e^{-k2 t}) (+) Poisson(k1(1-e^{-k2 t})/k2)."""
    check_birth_death_law(orc())


def check_gene_expression_moments(o, n=20000):
    km, gm, kp, gp = 2.0, 1.0, 5.0, 0.5
    states, _, status = o.ssa_paths(GE, [km, gm, kp, gp], [0, 0], [40.0], n, seed=78)
    assert (status == 0).all()
    m = states[:, 0, 0]
    p = states[:, 0, 1].astype(float)
    # stationary mRNA ~ Poisson(km/gm)
    assert chi2_pvalue(m, stats.poisson.pmf(np.arange(40), km / gm)) > 1e-3
    mean_p = km * kp / (gm * gp)
    fano_p = 1.0 + kp / (gm + gp)
    se = np.sqrt(fano_p * mean_p / n)
    assert abs(p.mean() - mean_p) < 5 * se
    assert abs(p.var() / p.mean() - fano_p) < 0.06 * fano_p


def test_ssa_gene_expression_stationary_moments():
    """mRNA ~ Poisson(k_m/g_m); protein mean k_m k_p/(g_m g_p), Fano 1 + k_p/(g_m+g_p)."""
    check_gene_expression_moments(orc())


def check_second_order_convention(o, n=20000):
    c, t = 0.3, 0.5
    s, _, _ = o.ssa_paths(DIMER, [c], [4], [t], n, seed=79)
    p_hat = np.mean(s[:, 0, 0] == 4)
    p = np.exp(-c * 6 * t)                       # h = C(4,2) = 6
    assert abs(p_hat - p) < 5 * np.sqrt(p * (1 - p) / n)
    c2 = 0.1
    s, _, _ = o.ssa_paths(HETERO, [c2], [3, 5, 0], [1.0], n, seed=80)
    p_hat = np.mean(s[:, 0, 2] == 0)
    p = np.exp(-c2 * 15 * 1.0)                   # h = 3 * 5
    assert abs(p_hat - p) < 5 * np.sqrt(p * (1 - p) / n)
    # every dimerisation removes two molecules: parity of the count is kept
    s, _, _ = o.ssa_paths(DIMER, [c], [7], [0.2, 1.0, 5.0], 2000, seed=81)
    assert (s % 2 == 1).all() and (s >= 1).all()


def test_ssa_second_order_mass_action_convention():
    """Gillespie's combinatorial propensity: X+X uses C(x,2), A+B uses x_A x_B."""
    check_second_order_convention(orc())


def test_ssa_conservation_and_nonnegativity():
    """A + B <-> C conserves A + C and B + C on every path; counts stay >= 0."""
    s, fired, _ = orc().ssa_paths(REVERSIBLE, [0.05, 1.0], [30, 20, 5],
                                  np.linspace(0.1, 5.0, 25), 500, seed=82)
    assert (s >= 0).all()
    assert (s[..., 0] + s[..., 2] == 35).all()
    assert (s[..., 1] + s[..., 2] == 25).all()
    assert fired.min() > 0


# ----------------------------------------------------------- resampling ---
def check_resampling(o):
    rng = np.random.default_rng(5)
    for N in [1, 2, 3, 7, 64, 1000]:
        # equal weights give the identity map for any uniform
        for r64 in [0, 1, 2**63, 2**64 - 1, int(rng.integers(0, 2**63))]:
            assert (o.resample_systematic(np.full(N, 2**32, np.uint64), r64) == np.arange(N)).all()
        for trial in range(20):
            q = rng.integers(0, 2**32 + 1, size=N).astype(np.uint64)
            q[rng.random(N) < 0.3] = 0
            q[rng.integers(N)] = 2**32
            r64 = int(rng.integers(0, 2**63)) * 2 + int(rng.integers(0, 2))
            a = o.resample_systematic(q, r64)
            assert len(a) == N and (np.diff(a) >= 0).all()
            assert (q[a] > 0).all()                                # zero weight never chosen
            counts = np.bincount(a, minlength=N)
            W_ = float(q.astype(np.float64).sum())
            expct = N * q.astype(np.float64) / W_
            assert (counts >= np.floor(expct - 1e-9)).all()
            assert (counts <= np.ceil(expct + 1e-9)).all()
    # the first systematic point sits at u = 0 when the word is 0: a leading
    # zero-weight particle must still be skipped
    q = np.array([0, 5, 0, 7], np.uint64)
    a = o.resample_systematic(q, 0)
    assert (q[a] > 0).all()
    # a single nonzero weight takes every slot
    q = np.zeros(9, np.uint64)
    q[4] = 12345
    assert (o.resample_systematic(q, 2**40) == 4).all()
    # unbiased: mean offspring over a uniform grid of the 64-bit word is N q_i / W
    q = np.array([1, 2, 3, 4, 5, 6, 7, 100], np.uint64) * 2**20
    N = len(q)
    tot = np.zeros(N)
    G = 4096
    for g in range(G):
        r64 = (g * 2**64) // G + 12345
        tot += np.bincount(o.resample_systematic(q, r64), minlength=N)
    assert np.allclose(tot / G, N * q / q.sum(), atol=2e-3)


def test_resampling_systematic_properties():
    check_resampling(orc())


# -------------------------------------------------- weight / likelihood ---
def check_weights_c_zero(o):
    """C = 0: every particle has the same weight; ll = sum_k log N(y_k; 0, sigma^2)."""
    rng = np.random.default_rng(9)
    K, P = 6, 2
    y = rng.normal(size=(2, K, P)) * 3.0
    sigma = np.array([1.5, 0.7])
    C = np.zeros((P, 2))
    want = stats.norm.logpdf(y, 0.0, sigma[None, None, :]).sum(axis=(1, 2))
    for N, seed in [(1, 1), (5, 2), (37, 3)]:
        r = o.pf_loglik(GE, [[0.5, 0.2, 2.0, 0.1]], [3, 4], np.arange(1, K + 1) * 0.7, y, C,
                        sigma, N, seed)
        assert np.allclose(r["ll_traj"][0], want, rtol=1e-13, atol=1e-12)
        assert np.isclose(r["loglik"][0], want.sum(), rtol=1e-13)


def test_weights_closed_form_when_C_zero():
    check_weights_c_zero(orc())


def check_single_particle(o):
    """N = 1: the filter never reweights anything away, so
    ll = sum_k log N(y_k; C x(t_k), diag sigma^2) along the particle's own path,
    which the simulator reproduces from the same counter keys."""
    rng = np.random.default_rng(10)
    theta = [0.8, 0.3, 3.0, 0.2]
    times = np.array([0.5, 1.5, 2.0, 4.0, 7.5])
    K, P = len(times), 2
    C = np.array([[1.0, 2.0], [0.5, -1.0]])       # not symmetric: catches a transpose
    sigma = np.array([2.0, 0.5])
    y = rng.normal(size=(1, K, P)) * 4.0 + 5.0
    r = o.pf_loglik(GE, [theta], [2, 1], times, y, C, sigma, 1, 4242, want_final_states=True)
    # the simulator's path 0 uses the same counters as particle 0 of trajectory 0, theta 0
    s, _, _ = o.ssa_paths(GE, theta, [2, 1], times, 1, seed=4242)
    xk = s[0].astype(float)                         # [K][U]
    mu = xk @ C.T                                   # [K][P]
    want = stats.norm.logpdf(y[0], mu, sigma[None, :]).sum()
    assert np.isclose(r["loglik"][0], want, rtol=1e-13)
    assert (r["final_states"][0, 0, 0] == s[0, -1]).all()


def test_single_particle_filter_is_path_likelihood():
    check_single_particle(o=orc())


def test_observation_at_time_zero():
    """obs_times[0] = 0: nothing is simulated, every particle sits at x0."""
    y = np.array([[[3.3]]])
    r = orc().pf_loglik(BD, [[10.0, 0.2]], [2], [0.0], y, [[1.0]], [1.7], 50, 1)
    assert np.isclose(r["loglik"][0], stats.norm.logpdf(3.3, 2.0, 1.7), rtol=1e-14)
    assert r["events"][0, 0] == 0


# ------------------------------------------------------ whole filter ------
def check_unbiased(o, S=400, N=200):
    """E[p_hat] = p (bootstrap-filter unbiasedness); Jensen: E[log p_hat] <= log p."""
    w = W.birth_death()
    y = w.observations()
    for (k1, k2) in [(10.0, 0.2), (14.0, 0.3)]:
        L, leak = exact_bd.loglik(k1, k2, 10, w.obs_times, y[0, :, 0], 1.0, 1.0, 200)
        assert abs(leak) < 1e-12
        lls = np.array([o.pf_loglik(w.net, [[k1, k2]], w.x0, w.obs_times, y, w.C, w.sigma, N,
                                    9000 + s)["loglik"][0] for s in range(S)])
        z = np.exp(lls - L)
        se = z.std(ddof=1) / np.sqrt(S)
        assert abs(z.mean() - 1.0) < 4 * se + 1e-3, (k1, k2, z.mean(), se)
        assert lls.mean() <= L + 4 * lls.std(ddof=1) / np.sqrt(S)


def test_filter_unbiased_against_exact_birth_death():
    check_unbiased(orc())


def test_filter_consistency_in_particle_count():
    """|log p_hat - log p| shrinks as N grows (filter consistency)."""
    w = W.birth_death()
    y = w.observations()
    L, _ = exact_bd.loglik(10.0, 0.2, 10, w.obs_times, y[0, :, 0], 1.0, 1.0, 200)
    err = {}
    for N in [20, 200, 2000]:
        lls = np.array([orc().pf_loglik(w.net, [[10.0, 0.2]], w.x0, w.obs_times, y, w.C,
                                        w.sigma, N, 500 + s)["loglik"][0] for s in range(12)])
        err[N] = np.sqrt(np.mean((lls - L) ** 2))
    # the error of log p_hat falls roughly like N^-1/2 (a factor ~3.2 per decade)
    assert err[200] < 0.5 * err[20]
    assert err[2000] < 0.5 * err[200]


# ------------------------------------ model extensions (Lac-Gfp forms) ----
# Birth-death with k1 composed as theta_0 + 3 theta_1 and k2 = theta_2, the
# initial count uniform on 5..15, and y ~ N(2 + 1.5 x, 1 + 0.5 x): the exact
# forward algorithm handles each extension in its own plain form.
MODEL = {"rate_coef": [[1.0, 3.0, 0.0], [0.0, 0.0, 1.0]], "x0_hi": [15], "obs_offset": [2.0],
         "obs_var": [[0.5]]}


def model_data():
    w = W.birth_death()
    xs, _, _ = orc().ssa_paths(BD, [10.0, 0.2], [9], w.obs_times, 1, seed=7070)
    xk = xs[0, :, 0].astype(float)
    rng = np.random.default_rng(77)
    y = 2.0 + 1.5 * xk + rng.normal(size=len(xk)) * np.sqrt(1.0 + 0.5 * xk)
    return w, y[None, :, None]


def check_model_unbiased(o, S=300, N=200):
    """E[p_hat] = p and Jensen for the extended model, against the exact
    likelihood of the same model (composed rate, uniform x0, affine variance)."""
    w, y = model_data()
    for th, (k1, k2) in [([4.0, 2.0, 0.2], (10.0, 0.2)), ([8.0, 2.0, 0.3], (14.0, 0.3))]:
        L, leak = exact_bd.loglik(k1, k2, 5, w.obs_times, y[0, :, 0], c=1.5, sigma=1.0, nmax=200,
                                  x0_hi=15, obs_offset=2.0, obs_var=0.5)
        assert abs(leak) < 1e-12
        lls = np.array([o.pf_loglik(BD, [th], [5], w.obs_times, y, [[1.5]], [1.0], N, 6100 + s,
                                    model=MODEL)["loglik"][0] for s in range(S)])
        z = np.exp(lls - L)
        se = z.std(ddof=1) / np.sqrt(S)
        assert abs(z.mean() - 1.0) < 4 * se + 1e-3, (th, z.mean(), se)
        assert lls.mean() <= L + 4 * lls.std(ddof=1) / np.sqrt(S)


def test_extended_model_unbiased_against_exact():
    check_model_unbiased(orc())


def check_initial_uniform(o, n=16384):
    """Initial particles of a random x0: each species uniform on its integers
    lo..hi (chi-square), species independent (correlations), filters
    (trajectories) independent.  Observation at t = 0: no simulation, so the
    final states are the initial draws."""
    net = W.cascade_network()
    U = net["reactants"].shape[1]
    R = net["reactants"].shape[0]
    lo = np.arange(U, dtype=np.int32)
    hi = lo + np.array([0, 1, 2, 3, 4, 5, 6, 7, 9, 30], np.int32)[:U]
    T = 2
    y = np.zeros((T, 1, 1))
    C = np.zeros((1, U))
    r = o.pf_loglik(net, np.ones((1, R)), lo, [0.0], y, C, [1.0], n, 31337,
                    want_final_states=True, model={"x0_hi": hi})
    fs = r["final_states"][0].astype(np.int64)            # [T][N][U]
    for t in range(T):
        X = fs[t]
        for u in range(U):
            span = int(hi[u] - lo[u] + 1)
            assert X[:, u].min() >= lo[u] and X[:, u].max() <= hi[u]
            if span == 1:
                continue
            cnt = np.bincount(X[:, u] - lo[u], minlength=span)
            assert cnt.min() > 0
            assert stats.chisquare(cnt).pvalue > 1e-4, (t, u, cnt)
        Z = (X[:, 1:] - X[:, 1:].mean(0)) / X[:, 1:].std(0)
        cor = (Z.T @ Z) / n - np.eye(U - 1)
        assert np.abs(cor).max() < 5 / np.sqrt(n)
    a = (fs[0, :, 9] - fs[0, :, 9].mean()) / fs[0, :, 9].std()
    b = (fs[1, :, 9] - fs[1, :, 9].mean()) / fs[1, :, 9].std()
    assert abs(np.mean(a * b)) < 5 / np.sqrt(n)


def test_random_initial_state_uniform():
    check_initial_uniform(orc())


def test_extended_observation_reduces_to_basic():
    """obs_var = 0 and obs_offset = 0 give the basic model's likelihood (the
    log-weights differ by the constant sum_p log sigma_p moved out of the
    normaliser, so values agree to rounding; resampling draws may differ only
    through the 2^-20 grid of the quantised weights, which equal weights do
    not feel: C = 0 makes all weights equal)."""
    rng = np.random.default_rng(5)
    y = rng.normal(size=(1, 6, 1)) * 2.0
    base = orc().pf_loglik(GE, [[0.5, 0.2, 2.0, 0.1]], [3, 4], np.arange(1, 7) * 0.5, y,
                           [[0.0, 0.0]], [1.3], 40, 8)
    ext = orc().pf_loglik(GE, [[0.5, 0.2, 2.0, 0.1]], [3, 4], np.arange(1, 7) * 0.5, y,
                          [[0.0, 0.0]], [1.3], 40, 8,
                          model={"obs_var": [[0.0, 0.0]], "obs_offset": [0.0]})
    assert np.isclose(base["loglik"][0], ext["loglik"][0], rtol=1e-13)
    assert (base["digest"] == ext["digest"]).all()


def test_composed_rates_reproduce_plain_rates():
    """Composition with one unit coefficient per reaction is the plain rate
    lookup, bit for bit (x + 0 and 1 * theta are exact)."""
    w = W.gene_expression()
    th = w.thetas(3)
    rc = np.eye(4)
    a = orc().pf_loglik(w.net, th, w.x0, w.obs_times[:5], w.observations()[:2, :5], w.C, w.sigma,
                        30, 4)
    b = orc().pf_loglik(w.net, th, w.x0, w.obs_times[:5], w.observations()[:2, :5], w.C, w.sigma,
                        30, 4, model={"rate_coef": rc})
    assert (a["loglik"] == b["loglik"]).all() and (a["digest"] == b["digest"]).all()


# ------------------------------------------------------- bookkeeping ------
def test_theta_ids_reproduce_batch_rows():
    w = W.birth_death()
    th = w.thetas(12)
    full = orc().pf_loglik(w.net, th, w.x0, w.obs_times, w.observations(), w.C, w.sigma, 30, 5)
    pick = np.array([3, 7, 11])
    sub = orc().pf_loglik(w.net, th[pick], w.x0, w.obs_times, w.observations(), w.C, w.sigma,
                          30, 5, theta_ids=pick)
    assert (sub["loglik"] == full["loglik"][pick]).all()
    assert (sub["digest"] == full["digest"][pick]).all()


def test_budget_marks_theta_minus_inf():
    w = W.birth_death()
    r = orc().pf_loglik(w.net, w.thetas(4), w.x0, w.obs_times, w.observations(), w.C, w.sigma,
                        10, 5, budget=3)
    assert (r["status"] == pf_oracle.BUDGET).all()
    assert np.isneginf(r["loglik"]).all()


def test_absorbing_network_fires_nothing():
    """All propensities zero (X -> 0 from x = 0): states stay, no draws are made."""
    r = orc().pf_loglik({"reactants": [[1]], "products": [[0]], "rate_index": None}, [[1.0]],
                        [0], [1.0, 2.0], np.array([[[0.5], [-0.2]]]), [[1.0]], [1.0], 8, 3)
    assert r["events"][0, 0] == 0
    want = stats.norm.logpdf([0.5, -0.2], 0.0, 1.0).sum()
    assert np.isclose(r["loglik"][0], want, rtol=1e-14)


def test_invalid_networks_rejected():
    with pytest.raises(ValueError):        # total order 3
        orc().pf_loglik({"reactants": [[3]], "products": [[0]], "rate_index": None}, [[1.0]],
                        [5], [1.0], np.zeros((1, 1, 1)), [[1.0]], [1.0], 4, 1)
    with pytest.raises(ValueError):        # rate index out of range
        orc().pf_loglik({"reactants": [[1]], "products": [[0]], "rate_index": [2]}, [[1.0]],
                        [5], [1.0], np.zeros((1, 1, 1)), [[1.0]], [1.0], 4, 1)


# --------------------------------------------------------------------------
# log-weight rounding and integer weights of the resampling step
# --------------------------------------------------------------------------
def nearest_multiple_2m20(e: float) -> float:
    """The multiple of 2^-20 nearest to e, ties to the even multiple, in
    exact rational arithmetic (Python's round() of a Fraction is
    round-half-even)."""
    from fractions import Fraction
    return float(Fraction(round(Fraction(e) * 2**20), 2**20))


def check_grid20(o):
    u = 2.0 ** -20
    cases = {0.0: 0.0, 3 * u: 3 * u, -7 * u: -7 * u,            # already on the grid
             0.5 * u: 0.0, 1.5 * u: 2 * u, 2.5 * u: 2 * u,    # ties go to the even multiple
             -0.5 * u: 0.0, -1.5 * u: -2 * u, -2.5 * u: -2 * u,
             0.3 * u: 0.0, 0.7 * u: u, -0.7 * u: -u,          # plain rounding
             1.0 / 3.0: 349525 * u, -1234.5: -1234.5}
    e = np.array(list(cases))
    got = o.grid20(e)
    assert np.array_equal(got, np.array(list(cases.values()))), (e, got)
    assert np.signbit(o.grid20([-0.5 * u])[0]) or o.grid20([-0.5 * u])[0] == 0.0
    rng = np.random.default_rng(20)
    r = np.concatenate([rng.normal(0, 3, 2000), rng.normal(0, 1e4, 500),
                        (rng.integers(-2**30, 2**30, 500) + 0.5) * u])   # many exact ties
    want = np.array([nearest_multiple_2m20(float(x)) for x in r])
    assert np.array_equal(o.grid20(r), want)


def test_grid20_is_round_to_nearest_multiple_of_2m20_ties_even():
    check_grid20(pf_oracle.default())


def check_quantised_weights(o):
    """q_i = floor(2^32 exp(e_i - max e)); with the state-dependent variance,
    from the rounded log-weights.  Exact facts: the maximal particle gets 2^32
    in either mode (also when max e is off the grid); two log-weights in the
    same 2^-20 cell get equal weights only in the rounded mode; exp(-2^-23)
    rounds to 1 - 2^-23 + 2^-47, so its weight is 2^32 - 512."""
    e = np.array([-1.0, -1.0 - 2.0 ** -23])
    assert list(o.quantise_weights(e, svar=False)) == [2**32, 2**32 - 512]
    assert list(o.quantise_weights(e, svar=True)) == [2**32, 2**32]
    off = np.array([-1.0 / 3.0, -0.3, -2.0])              # maximum -0.3, off the grid
    for svar in (False, True):
        q = o.quantise_weights(off, svar=svar)
        assert q[1] == 2**32 and q[0] < 2**32 and q[2] < q[0]
    q = o.quantise_weights(np.array([0.0, np.log(0.5)]), svar=False)
    assert q[0] == 2**32 and q[1] in (2**31, 2**31 - 1)
    # the first maximum in particle order is the reference
    assert list(o.quantise_weights(np.array([-0.5, -0.5]), svar=True)) == [2**32, 2**32]


def test_quantised_resampling_weights():
    check_quantised_weights(pf_oracle.default())
