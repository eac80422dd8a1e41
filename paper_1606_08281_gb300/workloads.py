"""Seeded synthetic workloads: networks, parameter batches and observations.

This module holds no arithmetic of the likelihood method itself.  It builds
network descriptions (stoichiometry tables), draws candidate parameter vectors
theta from log-uniform priors, and loads the stored observed trajectories.  The
observed trajectories ``y`` are inputs; they were written once by
``tests/golden/make_observations.py`` (which simulates the network at a fixed
theta* with the test oracle and adds Gaussian noise) and are read here from
``tests/golden/observations.json``.

Networks follow the paper's notation (Sec. "Chemical Reaction Networks"):
reaction r consumes p_ru and produces q_ru molecules of species u; its rate
constant is theta[rate_index[r]].  Shapes:
  reactants, products: int32 [R][U]; rate_index: int32 [R] or None (= r).

Workloads (sizes (U, R, P, K, T, M, N)):
  birth_death     (1, 2, 1, 20, 1, 200, 100)
  gene_expression (2, 4, 1, 50, 10, 4096, 1000)
  cascade         (10, 20, 3, 100, 16, 16384, 512)
"""
from __future__ import annotations

import json
from dataclasses import dataclass, field
from pathlib import Path

import numpy as np

REPO_ROOT = Path(__file__).resolve().parent.parent
OBSERVATIONS_PATH = REPO_ROOT / "tests" / "golden" / "observations.json"


# --------------------------------------------------------------------------
# networks
# --------------------------------------------------------------------------
def birth_death_network() -> dict:
    """0 -> X (k1), X -> 0 (k2 x): the paper's birth-death example."""
    return {
        "name": "birth_death",
        "species": ["X"],
        "reactants": np.array([[0], [1]], np.int32),
        "products": np.array([[1], [0]], np.int32),
        "rate_index": None,
    }


def gene_expression_network() -> dict:
    """Two-stage gene expression: 0->M (k_m), M->0 (g_m M), M->M+P (k_p M), P->0 (g_p P)."""
    return {
        "name": "gene_expression",
        "species": ["mRNA", "protein"],
        "reactants": np.array([[0, 0], [1, 0], [1, 0], [0, 1]], np.int32),
        "products": np.array([[1, 0], [0, 0], [1, 1], [0, 0]], np.int32),
        "rate_index": None,
    }


def telegraph_network() -> dict:
    """The RNA model of Supp. "Verification of approximated posterior":
    G_off -> G_on (theta_1), G_on -> G_off (theta_2), G_on -> G_on + RNA
    (theta_3), RNA -> 0 (theta_4)."""
    return {
        "name": "telegraph",
        "species": ["G_on", "G_off", "RNA"],
        "reactants": np.array([[0, 1, 0], [1, 0, 0], [1, 0, 0], [0, 0, 1]], np.int32),
        "products": np.array([[1, 0, 0], [0, 1, 0], [1, 0, 1], [0, 0, 0]], np.int32),
        "rate_index": None,
    }


def cascade_network(seed: int = 3000, U: int = 10, n0: int = 4, n1: int = 10, n2: int = 6) -> dict:
    """Seeded synthetic signalling cascade with mass-action orders <= 2.

    Rules: every species is consumed by one first-order reaction that either
    converts it into the next species of a random chain or degrades it (the
    chain's last species always degrades, so every species drains); order-2
    reactions A + B -> C or A + B -> 0 conserve or destroy mass; order-0
    reactions produce one molecule.  Every species is a product of at least one
    reaction.  Returns the network plus the rate bounds per reaction.
    """
    rng = np.random.default_rng(seed)
    R = n0 + n1 + n2
    assert n1 == U, "one first-order reaction per species"
    reac = np.zeros((R, U), np.int32)
    prod = np.zeros((R, U), np.int32)
    order = np.zeros(R, np.int32)
    r = 0
    for _ in range(n0):                                # 0 -> X_v
        prod[r, rng.integers(U)] = 1
        order[r] = 0
        r += 1
    chain = rng.permutation(U)
    for i, u in enumerate(chain):                      # X_u -> X_next or X_u -> 0
        reac[r, u] = 1
        if i + 1 < U and rng.random() < 0.6:
            prod[r, chain[i + 1]] = 1
        order[r] = 1
        r += 1
    for _ in range(n2):                                # X_a + X_b -> X_c or -> 0
        a, b = rng.integers(U), rng.integers(U)
        reac[r, a] += 1
        reac[r, b] += 1
        if rng.random() < 0.7:
            prod[r, rng.integers(U)] = 1
        order[r] = 2
        r += 1
    # repair: every species must be produced by some reaction
    for u in range(U):
        if prod[:, u].sum() == 0:
            cands = [rr for rr in range(R) if order[rr] in (0, 2)]
            rr = cands[int(rng.integers(len(cands)))]
            prod[rr, :] = 0
            prod[rr, u] = 1
    for u in range(U):
        assert reac[:, u].sum() > 0 and prod[:, u].sum() > 0
    bounds = {0: (0.1, 100.0), 1: (1e-3, 1.0), 2: (1e-5, 1e-2)}
    lo = np.array([bounds[int(o)][0] for o in order])
    hi = np.array([bounds[int(o)][1] for o in order])
    return {
        "name": "cascade",
        "species": [f"S{u}" for u in range(U)],
        "reactants": reac,
        "products": prod,
        "rate_index": None,
        "order": order,
        "prior_lo": lo,
        "prior_hi": hi,
    }


LAC_GFP_SPECIES = ["lacI", "LACI", "LACI2", "PLac", "O2Lac", "O4Lac", "gfp", "GFP", "mGFP"]
IPTG_uM = 10.0


def lac_gfp_network() -> dict:
    """The Lac-Gfp network of Supp. "LacGfp example": 9 species, 18 mass-action
    reactions, 18 parameters.  Reaction 4 (LACI degradation) has the composed
    rate theta_4 + theta_5 [IPTG] with [IPTG] = 10 uM; reaction 18 (mGFP
    degradation) shares theta_17 with reaction 16 (GFP degradation).  The
    rates are given by `rate_coef` [R][d] (pf_model)."""
    ix = {s: i for i, s in enumerate(LAC_GFP_SPECIES)}
    rx = [({}, {"lacI": 1}),                                    # 1  theta_1
          ({"lacI": 1}, {}),                                    # 2  theta_2
          ({"lacI": 1}, {"lacI": 1, "LACI": 1}),                # 3  theta_3
          ({"LACI": 1}, {}),                                    # 4  theta_4 + theta_5 [IPTG]
          ({"LACI": 2}, {"LACI2": 1}),                          # 5  theta_6
          ({"LACI2": 1}, {"LACI": 2}),                          # 6  theta_7
          ({"LACI2": 1, "PLac": 1}, {"O2Lac": 1}),              # 7  theta_8
          ({"O2Lac": 1}, {"LACI2": 1, "PLac": 1}),              # 8  theta_9
          ({"O2Lac": 2}, {"O4Lac": 1}),                         # 9  theta_10
          ({"O4Lac": 1}, {"O2Lac": 2}),                         # 10 theta_11
          ({"PLac": 1}, {"PLac": 1, "gfp": 1}),                 # 11 theta_12
          ({"O2Lac": 1}, {"O2Lac": 1, "gfp": 1}),               # 12 theta_13
          ({"O4Lac": 1}, {"O4Lac": 1, "gfp": 1}),               # 13 theta_14
          ({"gfp": 1}, {}),                                     # 14 theta_15
          ({"gfp": 1}, {"gfp": 1, "GFP": 1}),                   # 15 theta_16
          ({"GFP": 1}, {}),                                     # 16 theta_17
          ({"GFP": 1}, {"mGFP": 1}),                            # 17 theta_18
          ({"mGFP": 1}, {})]                                    # 18 theta_17
    R, U = len(rx), len(LAC_GFP_SPECIES)
    reac = np.zeros((R, U), np.int32)
    prod = np.zeros((R, U), np.int32)
    for r, (a, b) in enumerate(rx):
        for k, v in a.items():
            reac[r, ix[k]] = v
        for k, v in b.items():
            prod[r, ix[k]] = v
    cols = [0, 1, 2, None, 5, 6, 7, 8, 9, 10, 11, 12, 13, 14, 15, 16, 17, 16]
    rate_coef = np.zeros((R, 18))
    for r, c in enumerate(cols):
        if c is None:
            rate_coef[r, 3] = 1.0
            rate_coef[r, 4] = IPTG_uM
        else:
            rate_coef[r, c] = 1.0
    return {"name": "lac_gfp", "species": LAC_GFP_SPECIES, "reactants": reac, "products": prod,
            "rate_index": None, "rate_coef": rate_coef}


# --------------------------------------------------------------------------
# parameter draws
# --------------------------------------------------------------------------
def log_uniform(rng: np.random.Generator, lo, hi, M: int) -> np.ndarray:
    """M rows of independent log-uniform draws between lo[i] and hi[i]."""
    lo = np.log(np.asarray(lo, float))
    hi = np.log(np.asarray(hi, float))
    return np.exp(rng.uniform(lo, hi, size=(M, len(lo))))


# --------------------------------------------------------------------------
# workloads
# --------------------------------------------------------------------------
@dataclass
class Workload:
    name: str
    net: dict
    x0: np.ndarray            # int32 [U]
    obs_times: np.ndarray     # float64 [K]
    C: np.ndarray             # float64 [P][U]
    sigma: np.ndarray         # float64 [P]
    prior_lo: np.ndarray      # float64 [d]
    prior_hi: np.ndarray      # float64 [d]
    theta_star: np.ndarray    # float64 [d] (data-generating)
    T: int
    M: int
    N: int
    theta_seed: int
    filter_seed: int
    data_seed: int
    y: np.ndarray | None = field(default=None)   # float64 [T][K][P]
    model: dict | None = field(default=None)     # pf_model extensions (None: basic model)
    fsp_box: np.ndarray | None = field(default=None)  # int32 [U] box of the exact (FSP) likelihood

    @property
    def U(self) -> int:
        return int(self.net["reactants"].shape[1])

    @property
    def R(self) -> int:
        return int(self.net["reactants"].shape[0])

    @property
    def K(self) -> int:
        return int(len(self.obs_times))

    @property
    def P(self) -> int:
        return int(self.C.shape[0])

    def thetas(self, M: int | None = None) -> np.ndarray:
        """The workload's seeded theta batch (first M rows of the full batch)."""
        rng = np.random.default_rng(self.theta_seed)
        full = log_uniform(rng, self.prior_lo, self.prior_hi, self.M)
        return np.ascontiguousarray(full[: (self.M if M is None else M)])

    def observations(self) -> np.ndarray:
        if self.y is None:
            self.y = load_observations(self.name)
        return self.y

    def subset(self, T: int | None = None, K: int | None = None) -> "Workload":
        """A copy restricted to the first T trajectories and first K observation times."""
        T = self.T if T is None else T
        K = self.K if K is None else K
        w = Workload(**{**self.__dict__})
        w.T = T
        w.obs_times = self.obs_times[:K].copy()
        w.y = self.observations()[:T, :K, :].copy()
        return w


def birth_death() -> Workload:
    return Workload(
        name="birth_death", net=birth_death_network(), x0=np.array([10], np.int32),
        obs_times=np.arange(1, 21, dtype=np.float64), C=np.array([[1.0]]),
        sigma=np.array([1.0]), prior_lo=np.array([1.0, 0.05]), prior_hi=np.array([50.0, 1.0]),
        theta_star=np.array([10.0, 0.2]), T=1, M=200, N=100,
        data_seed=1001, theta_seed=1002, filter_seed=1003, fsp_box=np.array([1200], np.int32))


def gene_expression() -> Workload:
    ts = np.array([0.1, 0.1, 1.0, 0.01])
    return Workload(
        name="gene_expression", net=gene_expression_network(), x0=np.array([0, 0], np.int32),
        obs_times=5.0 * np.arange(1, 51, dtype=np.float64), C=np.array([[0.0, 1.0]]),
        sigma=np.array([5.0]), prior_lo=ts / 10.0, prior_hi=ts * 10.0, theta_star=ts, T=10, M=4096, N=1000,
        data_seed=2001, theta_seed=2002, filter_seed=2003)


def cascade() -> Workload:
    net = cascade_network(3000)
    rng = np.random.default_rng(3004)
    x0 = rng.integers(0, 101, size=10).astype(np.int32)
    theta_star = log_uniform(np.random.default_rng(3005), net["prior_lo"], net["prior_hi"], 1)[0]
    C = np.zeros((3, 10))
    C[0, 0] = C[1, 1] = C[2, 2] = 1.0
    return Workload(
        name="cascade", net=net, x0=x0, obs_times=np.arange(1, 101, dtype=np.float64), C=C,
        sigma=np.array([2.0, 2.0, 2.0]), prior_lo=net["prior_lo"], prior_hi=net["prior_hi"],
        theta_star=theta_star, T=16, M=16384, N=512,
        data_seed=3001, theta_seed=3002, filter_seed=3003)


# Lac-Gfp (Supp. "LacGfp example"): theta* and the log-uniform prior of the
# paper's table; theta_10's prior is printed as [0.16, 1.600] beside
# theta_10* = 173.576 and is read as [0.16, 1600].  Observation of mGFP:
# N(22.85 x, 5.72 sqrt(x)) plus a background; the paper's measured background
# distribution is not available, so a Gaussian N(100, 30^2) stands in.
LAC_GFP_THETA_STAR = np.array([1.215, 7.430, 1.439, 3.971, 1.173, 1716.683, 6.282, 0.433, 0.679,
                               173.576, 0.623, 119.232, 0.120, 0.006, 1.673, 32.318, 1.196,
                               2.102])
LAC_GFP_PRIOR = np.array([[1, 50], [0.1, 30], [1, 50], [0.1, 20], [1, 100], [0.16, 3000],
                          [0.1, 20], [0.0016, 1.6], [0.1, 20], [0.16, 1600], [0.1, 20], [1, 150],
                          [0.1, 15], [1e-5, 1], [0.1, 20], [1, 50], [0.1, 20], [0.1, 20]], float)
LAC_GFP_X0_LO = np.array([0, 0, 0, 0, 0, 50, 0, 0, 0], np.int32)
LAC_GFP_X0_HI = np.array([5, 10, 0, 0, 0, 70, 0, 0, 0], np.int32)
LAC_GFP_GAIN, LAC_GFP_NOISE = 22.85, 5.72
LAC_GFP_BACKGROUND = (100.0, 30.0)


def lac_gfp() -> Workload:
    net = lac_gfp_network()
    C = np.zeros((1, 9))
    C[0, 8] = LAC_GFP_GAIN
    V = np.zeros((1, 9))
    V[0, 8] = LAC_GFP_NOISE ** 2
    model = {"rate_coef": net["rate_coef"], "x0_hi": LAC_GFP_X0_HI,
             "obs_offset": np.array([LAC_GFP_BACKGROUND[0]]), "obs_var": V}
    return Workload(
        name="lac_gfp", net=net, x0=LAC_GFP_X0_LO.copy(),
        obs_times=np.arange(1, 30, dtype=np.float64), C=C,
        sigma=np.array([LAC_GFP_BACKGROUND[1]]), prior_lo=LAC_GFP_PRIOR[:, 0],
        prior_hi=LAC_GFP_PRIOR[:, 1], theta_star=LAC_GFP_THETA_STAR.copy(), T=4, M=256, N=200,
        data_seed=6001, theta_seed=6002, filter_seed=6003, model=model)


def telegraph() -> Workload:
    """The paper's RNA model: one trajectory of mRNA observed at 25 equally
    spaced times in (0, 200], theta_1 unknown (log-uniform prior
    [1e-6, 0.006]), theta_2..4 known.  The observation noise is not stated;
    read as RNA + N(0, 1).  Data seed 7003 is the first from 7001 on whose path
    switches the gene on within the 200 time units (theta_1* = 0.001 leaves the
    gene off in most paths, and then the data carry little information)."""
    ts = np.array([0.001, 0.002, 0.06, 0.002])
    lo = ts.copy()
    hi = ts.copy()
    lo[0], hi[0] = 1e-6, 0.006
    return Workload(
        name="telegraph", net=telegraph_network(), x0=np.array([0, 1, 0], np.int32),
        obs_times=8.0 * np.arange(1, 26, dtype=np.float64), C=np.array([[0.0, 0.0, 1.0]]),
        sigma=np.array([1.0]), prior_lo=lo, prior_hi=hi, theta_star=ts, T=1, M=4096, N=200,
        data_seed=7003, theta_seed=7101, filter_seed=7102,
        fsp_box=np.array([1, 1, 60], np.int32))


WORKLOADS = {"birth_death": birth_death, "gene_expression": gene_expression, "cascade": cascade,
             "lac_gfp": lac_gfp, "telegraph": telegraph}


# --------------------------------------------------------------------------
# the deterministic Egf-Ras-Raf-Mek-Erk model (ODE likelihood)
# --------------------------------------------------------------------------
# theta layout (36): 27 kinetic constants (k1, gamma1, k2, K2, gamma2, D2, k3,
# K3, K_NFB, gamma3, D3, k4, K4, gamma4, D4, k5, K5, gamma5, D5, k6, K6, K6R,
# gamma6, D6, dusp_basal, dusp_ind, K_dusp), the initial EGFR, NFB and
# dusp (= DUSP) concentrations, and the FRET model (bg, lam, sigma, E, f_AA,
# f_DD).  Priors as in the paper's tables: kinetic constants log-uniform on
# [e^-10, e^5], initial concentrations [e^-8, e^1], FRET bg and lam
# [e^-7, e^6], sigma [e^-8, e^-3], E [e^-4, e^-0.5], f_AA and f_DD [e^-8, e^5].
ERK_PRIOR_LO = np.exp(np.array([-10.0] * 27 + [-8.0] * 3 + [-7.0, -7.0, -8.0, -4.0, -8.0, -8.0]))
ERK_PRIOR_HI = np.exp(np.array([5.0] * 27 + [1.0] * 3 + [6.0, 6.0, -3.0, -0.5, 5.0, 5.0]))
# The data-generating parameters are not in the paper (its data are measured);
# this synthetic theta gives a FRET response of about 0.5 -> 0.8 with a slow
# Dusp feedback over two hours.
ERK_THETA_BAR = np.array([1.0, 0.1, 1.0, 0.5, 0.5, 0.5, 1.0, 0.5, 0.5, 0.5, 0.5, 1.0, 0.5, 0.5,
                          0.5, 1.0, 0.5, 5.0, 0.5, 0.5, 0.5, 0.5, 0.1, 0.5, 0.001, 100.0, 0.01,
                          1.0, 0.5, 0.001, 0.5, 1.0, 0.02, 0.3, 1.0, 1.0])


def _pulses(period: float, width: float, end: float = 120.0):
    st, sv, t = [], [], 0.0
    while t < end:
        st += [t, t + width]
        sv += [1.0, 0.0]
        t += period
    return np.array(st), np.array(sv)


def erk_patterns() -> list:
    """Six EGF input patterns (the paper's stimuli are not given): a sustained
    step, one 10-min pulse, 5-min pulses every 20 and every 40 min, 3-min pulses
    every 10 min, and two 20-min pulses an hour apart.  Each is (switch times,
    values): the input is values[i] from switch time i on."""
    return [(np.array([0.0]), np.array([1.0])), (np.array([0.0, 10.0]), np.array([1.0, 0.0])),
            _pulses(20.0, 5.0), _pulses(40.0, 5.0), _pulses(10.0, 3.0),
            (np.array([0.0, 20.0, 60.0, 80.0]), np.array([1.0, 0.0, 1.0, 0.0]))]


@dataclass
class ErkWorkload:
    name: str = "erk"
    theta_bar: np.ndarray = field(default_factory=lambda: ERK_THETA_BAR.copy())
    prior_lo: np.ndarray = field(default_factory=lambda: ERK_PRIOR_LO.copy())
    prior_hi: np.ndarray = field(default_factory=lambda: ERK_PRIOR_HI.copy())
    obs_times: np.ndarray = field(default_factory=lambda: 2.0 * np.arange(1, 61))
    M: int = 4096
    theta_seed: int = 8002
    data_seed: int = 8001
    y: np.ndarray | None = None

    @property
    def patterns(self) -> list:
        return erk_patterns()

    @property
    def K(self) -> int:
        return int(len(self.obs_times))

    def thetas(self, M: int | None = None, spread: float = 1.0) -> np.ndarray:
        """Log-uniform draws within a factor e^spread of theta_bar (clipped to
        the prior): a neighbourhood such as the sampler's later level sets."""
        lo = np.maximum(self.prior_lo, self.theta_bar * np.exp(-spread))
        hi = np.minimum(self.prior_hi, self.theta_bar * np.exp(spread))
        rng = np.random.default_rng(self.theta_seed)
        full = log_uniform(rng, lo, hi, self.M)
        return np.ascontiguousarray(full[: (self.M if M is None else M)])

    def prior_thetas(self, M: int, seed: int = 8003) -> np.ndarray:
        return log_uniform(np.random.default_rng(seed), self.prior_lo, self.prior_hi, M)

    def observations(self) -> np.ndarray:
        """[n_patterns][K] FRET observations."""
        if self.y is None:
            with open(OBSERVATIONS_PATH) as f:
                self.y = np.array(json.load(f)["erk"]["y"], dtype=np.float64)
        return self.y


def erk() -> ErkWorkload:
    return ErkWorkload()


def get(name: str) -> Workload:
    return WORKLOADS[name]()


def load_observations(name: str, path: Path = OBSERVATIONS_PATH) -> np.ndarray:
    with open(path) as f:
        data = json.load(f)
    return np.array(data[name]["y"], dtype=np.float64)


# --------------------------------------------------------------------------
# request mixes for the batching and serving patterns
# --------------------------------------------------------------------------
@dataclass
class RequestSpec:
    problem: str            # workload name
    thetas: np.ndarray      # [M][d]
    n_particles: int
    K_use: int
    seed: int
    arrival_s: float = 0.0
    threshold: float = float("nan")


def hetero_mix(seed: int = 4001, n_requests: int = 64, max_theta: int = 4096,
               max_theta_cascade: int = 4096, lac_gfp_rows: int = 32) -> list[RequestSpec]:
    """Heterogeneous batch (the batched-launch configuration): problems uniform
    over the three networks, theta counts log-uniform integers in
    [1, max_theta] ([1, max_theta_cascade] for the 10-species cascade),
    particle counts uniform over {256, 512, 1024, 2048, 4096}, observation
    prefix K uniform in [10, 100] capped at the problem's K; plus, when
    lac_gfp_rows > 0, one Lac-Gfp request (the paper's large stochastic
    example: the first lac_gfp_rows rows of its workload, all 4 trajectories,
    N = 200, K = 29)."""
    rng = np.random.default_rng(seed)
    names = ["birth_death", "gene_expression", "cascade"]
    wl = {n: get(n) for n in names}
    out = []
    for i in range(n_requests):
        name = names[int(rng.integers(3))]
        w = wl[name]
        hi = max_theta_cascade if name == "cascade" else max_theta
        M = int(np.floor(np.exp(rng.uniform(0.0, np.log(hi + 1)))))
        M = max(1, min(hi, M))
        N = int(rng.choice([256, 512, 1024, 2048, 4096]))
        K = min(w.K, int(rng.integers(10, 101)))
        th = log_uniform(rng, w.prior_lo, w.prior_hi, M)
        out.append(RequestSpec(name, th, N, K, int(seed * 1000 + i)))
    if lac_gfp_rows > 0:
        w = lac_gfp()
        out.append(RequestSpec("lac_gfp", w.thetas(lac_gfp_rows), w.N, w.K, int(seed * 1000 + n_requests)))
    return out


def serving_stream(seed: int = 5001, rate_hz: float = 200.0, duration_s: float = 10.0,
                   theta_range=(4, 512), cascade_theta_range=(1, 32)) -> list[RequestSpec]:
    """Poisson arrivals of level-set batches: a seeded coin picks the
    gene-expression or the cascade network; theta counts are log-uniform in
    the given ranges; N = 256 (gene expression, first 10 observation times) or
    128 (cascade, first 5).  Each request carries the median log-likelihood of
    the previous request of its network as its level-set threshold (the
    alpha = 50% quantile rule of the sampler), informational only."""
    rng = np.random.default_rng(seed)
    wl = {n: get(n) for n in ("gene_expression", "cascade")}
    t = 0.0
    out = []
    i = 0
    while True:
        t += rng.exponential(1.0 / rate_hz)
        if t > duration_s:
            break
        name = "gene_expression" if rng.random() < 0.5 else "cascade"
        w = wl[name]
        lo, hi = theta_range if name == "gene_expression" else cascade_theta_range
        M = int(np.clip(np.floor(np.exp(rng.uniform(np.log(lo), np.log(hi + 1)))), lo, hi))
        N, K = (256, 10) if name == "gene_expression" else (128, 5)
        th = log_uniform(rng, w.prior_lo, w.prior_hi, M)
        out.append(RequestSpec(name, th, N, K, int(seed * 100000 + i), arrival_s=t))
        i += 1
    return out
