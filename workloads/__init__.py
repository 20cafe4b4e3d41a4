"""Seeded synthetic inputs for the design-objective engine.

This module builds problem instances -- correlation matrices, mean shifts,
rejection thresholds, draw counts, stream keys and design Jacobians -- for
the five benchmark configurations.  It is the only code that both the CUDA
path and the FP64 oracle consume; it holds no estimator arithmetic (no
sampling, no probability evaluation).  Thresholds that satisfy the FWER
constraint of Eq. 2 are read from ``fwer_tables.json``, a stored table of
calibrated alpha scales written by ``oracle/make_fwer_tables.py``.

Design model (Sec. 2.1 Eq. 3; Sec. 3 Eq. 9-10; the cutoff / allocation
parametrisation is a reading of the benchmark configurations):
  r_i   = 1 - q (i-1)/(d-1)                    nested population fractions
  Delta = delta_plus - (delta_plus - delta_minus) r   hazard reduction
  theta = -log(1 - Delta)                      log hazard ratio
  mu_i  = sqrt(r_i I3) theta_i                 mean of the Z statistics
  w(a)  = (1 - a, a/(d-1), ..., a/(d-1)),  alpha = s(a) w,  b = Z_{1-alpha}
The design parameters are theta_design = (q, a, delta_plus, delta_minus); the
Jacobian dt/dtheta_design of t = b - mu is returned for the adjoint.
"""
import json
import math
import os

import numpy as np
from scipy import interpolate, special

HERE = os.path.dirname(os.path.abspath(__file__))
TABLE_PATH = os.path.join(HERE, "fwer_tables.json")

ALPHA0 = 0.025          # one-sided FWER level (Sec. 3, alpha = 0.025)
I3 = 211.0              # information units for Delta = 0.2 (Sec. 3)
A_RANGE = (0.2, 0.8)    # allocation fractions of the benchmark grids
Q_RANGE = (0.05, 0.95)  # cutoff quantiles of the benchmark grids
MAX_D = 20


# ------------------------------------------------------------------ tables
_TABLES = None


def tables():
    global _TABLES
    if _TABLES is None:
        if not os.path.exists(TABLE_PATH):
            raise FileNotFoundError("missing %s; run oracle/make_fwer_tables.py" % TABLE_PATH)
        with open(TABLE_PATH) as f:
            _TABLES = json.load(f)
    return _TABLES


class ScaleCurve:
    """alpha scale s(a) and ds/da by a cubic spline through a stored table."""

    def __init__(self, a, s):
        self.spline = interpolate.CubicSpline(np.asarray(a), np.asarray(s))
        self.lo, self.hi = float(a[0]), float(a[-1])

    def __call__(self, a):
        a = np.asarray(a, dtype=np.float64)
        if np.any(a < self.lo - 1e-12) or np.any(a > self.hi + 1e-12):
            raise ValueError("allocation outside the calibrated range")
        return self.spline(a), self.spline(a, 1)


# ----------------------------------------------------------- design model
def fractions(q, d):
    i = np.arange(d, dtype=np.float64)
    return 1.0 - q * i / (d - 1)


def alloc_weights(a, d):
    w = np.full(d, a / (d - 1))
    w[0] = 1.0 - a
    return w


def design_region(q, a, dp, dm, d, scale, dscale, I3=I3):
    """mu, b and dt/dtheta (d x 4, columns q, a, delta_plus, delta_minus)."""
    r = fractions(q, d)
    Delta = dp - (dp - dm) * r
    theta = -np.log1p(-Delta)
    sq = np.sqrt(r * I3)
    mu = sq * theta
    w = alloc_weights(a, d)
    alpha = scale * w
    b = special.ndtri(1.0 - alpha)
    # derivatives
    dr_dq = -np.arange(d, dtype=np.float64) / (d - 1)
    dtheta_dDelta = 1.0 / (1.0 - Delta)
    with np.errstate(divide="ignore", invalid="ignore"):
        dsq_dr = np.where(r > 0, 0.5 * math.sqrt(I3) / np.sqrt(r), 0.0)
    dmu_dr = dsq_dr * theta + sq * dtheta_dDelta * (-(dp - dm))
    dmu_dq = dmu_dr * dr_dq
    dmu_ddp = sq * dtheta_dDelta * (1.0 - r)
    dmu_ddm = sq * dtheta_dDelta * r
    dw_da = np.full(d, 1.0 / (d - 1))
    dw_da[0] = -1.0
    dalpha_da = dscale * w + scale * dw_da
    phi_b = np.exp(-0.5 * b * b) / math.sqrt(2.0 * math.pi)
    db_da = -dalpha_da / phi_b
    jac = np.stack([-dmu_dq, db_da, -dmu_ddp, -dmu_ddm], axis=1)
    return mu, b, jac


# ------------------------------------------------------------- structures
def equicorrelated(d, rho):
    return (1.0 - rho) * np.eye(d) + rho * np.ones((d, d))


def ar1(d, rho):
    i = np.arange(d)
    return rho ** np.abs(i[:, None] - i[None, :])


def block_equicorrelated(sizes, rho_in, rho_out):
    d = sum(sizes)
    S = np.full((d, d), rho_out)
    start = 0
    for n in sizes:
        S[start:start + n, start:start + n] = rho_in
        start += n
    np.fill_diagonal(S, 1.0)
    return S


def lkj_cvine(d, eta, rng):
    """Random correlation matrix with density proportional to det(R)^(eta-1),
    by the C-vine method of Lewandowski, Kurowicka and Joe (2009): on vine
    level k the partial correlations P[k, i] (i > k) are 2 Beta(b_k, b_k) - 1
    with b_k = eta + (d - 2 - k)/2, and each is turned into a correlation by
    the recursion over the lower levels l = k-1, ..., 0."""
    P = np.zeros((d, d))
    R = np.eye(d)
    beta = eta + (d - 1) / 2.0
    for k in range(d - 1):
        beta -= 0.5
        for i in range(k + 1, d):
            P[k, i] = 2.0 * rng.beta(beta, beta) - 1.0
            p = P[k, i]
            for l in range(k - 1, -1, -1):
                p = p * math.sqrt((1.0 - P[l, i] ** 2) * (1.0 - P[l, k] ** 2)) + P[l, i] * P[l, k]
            R[k, i] = R[i, k] = p
    return R


# ----------------------------------------------------------------- problem
class Problem:
    """Host-side (numpy) description of a batch of designs.

    Scenario s: dimension d_s, correlation matrix Sigma_s (d_s x d_s).
    Design j: scenario design_scen[j]; mu_j, b_j (d values each, packed in
    design order); n_draws[j]; draw_begin[j]; key[j] (stream key; equal keys
    within a scenario give common random numbers); optional Jacobian
    jac[j] (d x k) of t = b - mu with respect to the design parameters.
    """

    def __init__(self, name, sigmas, design_scen, mus, bs, n_draws, keys,
                 draw_begin=None, jacs=None, grid=None, structures=None, params=None):
        self.name = name
        self.sigmas = [np.ascontiguousarray(s, dtype=np.float64) for s in sigmas]
        self.scen_d = np.array([s.shape[0] for s in self.sigmas], dtype=np.int32)
        self.design_scen = np.asarray(design_scen, dtype=np.int32)
        self.mus = [np.asarray(m, dtype=np.float64) for m in mus]
        self.bs = [np.asarray(b, dtype=np.float64) for b in bs]
        self.n_draws = np.asarray(n_draws, dtype=np.uint64)
        self.keys = np.asarray(keys, dtype=np.uint64)
        J = len(self.mus)
        self.draw_begin = np.zeros(J, np.uint64) if draw_begin is None else np.asarray(draw_begin, np.uint64)
        self.jacs = jacs
        self.grid = grid              # (G1, G2) per scenario, or None
        self.structures = structures  # per scenario structure descriptors
        self.params = params          # per design (q, a, dp, dm) or None

    @property
    def n_scen(self):
        return len(self.sigmas)

    @property
    def n_design(self):
        return len(self.mus)

    def d_of(self, j):
        return int(self.scen_d[self.design_scen[j]])

    def sigma_packed(self):
        return np.concatenate([s.ravel() for s in self.sigmas])

    def mu_packed(self):
        return np.concatenate(self.mus) if self.mus else np.zeros(0)

    def b_packed(self):
        return np.concatenate(self.bs) if self.bs else np.zeros(0)

    def jac_packed(self):
        """[sum_j d_j * k] row-major per design (d x k)."""
        return np.concatenate([np.asarray(x, np.float64).ravel() for x in self.jacs])

    def t(self, j):
        return self.bs[j] - self.mus[j]

    def total_draws(self):
        return int(self.n_draws.sum())

    def subset(self, idx, name=None):
        idx = list(idx)
        return Problem(name or self.name + "-subset", self.sigmas, self.design_scen[idx],
                       [self.mus[j] for j in idx], [self.bs[j] for j in idx], self.n_draws[idx],
                       self.keys[idx], self.draw_begin[idx],
                       None if self.jacs is None else [self.jacs[j] for j in idx],
                       None, self.structures,
                       None if self.params is None else [self.params[j] for j in idx])


def _grid_problem(name, sigmas, structures, scen_params, curves, qs, as_, d, n_draws, keys):
    """Scenarios x (q grid) x (a grid), design index s*G1*G2 + iq*G2 + ia."""
    mus, bs, jacs, scen, params, key_list = [], [], [], [], [], []
    G1, G2 = len(qs), len(as_)
    for s, (dp, dm) in enumerate(scen_params):
        sc, dsc = curves[s](as_)
        for iq, q in enumerate(qs):
            for ia, a in enumerate(as_):
                mu, b, jac = design_region(q, a, dp, dm, d, float(sc[ia]), float(dsc[ia]))
                mus.append(mu); bs.append(b); jacs.append(jac); scen.append(s)
                params.append((float(q), float(a), float(dp), float(dm)))
                j = len(mus) - 1
                key_list.append(s if keys == "crn" else j)
    J = len(mus)
    return Problem(name, sigmas, scen, mus, bs, np.full(J, n_draws, np.uint64), key_list,
                   jacs=jacs, grid=(G1, G2), structures=structures, params=params)


# ---------------------------------------------------------------- configs
def c1(n_draws=100_000, keys="crn"):
    """d=3, rho=0.5 equicorrelated, 101 cutoff quantiles 0.05..0.95,
    delta+ = 0.5, delta- = 0.1, common critical value (equal alpha, FWER 0.025)."""
    t = tables()["c1"]
    d, rho = 3, t["rho"]
    b_star = float(special.ndtri(1.0 - t["scale"] / 3.0))
    qs = 0.05 + 0.009 * np.arange(101)
    mus, bs, params = [], [], []
    for q in qs:
        mu, _, _ = design_region(q, 2.0 / 3.0, 0.5, 0.1, d, t["scale"], 0.0)
        mus.append(mu)
        bs.append(np.full(d, b_star))
        params.append((float(q), None, 0.5, 0.1))
    J = len(qs)
    key_list = [0] * J if keys == "crn" else list(range(J))
    return Problem("c1", [equicorrelated(d, rho)], np.zeros(J, np.int32), mus, bs,
                   np.full(J, n_draws, np.uint64), key_list, grid=(1, J),
                   structures=[{"kind": "equi", "rho": rho}], params=params)


def c2_scenarios(n_scen=16, seed=0):
    """(delta+, delta-, rho) per scenario, drawn in that order from default_rng(seed)."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n_scen):
        dp = rng.uniform(0.3, 0.7)
        dm = rng.uniform(0.0, 0.2)
        rho = rng.uniform(0.2, 0.7)
        out.append((float(dp), float(dm), float(rho)))
    return out


def c2(n_scen=16, g1=64, g2=64, n_draws=1_000_000, keys="crn"):
    """d=3 grid of g1 cutoff quantiles x g2 allocations over 16 scenarios."""
    tab = tables()["c2"]["scenarios"]
    sc = c2_scenarios(16)[:n_scen]
    sigmas = [equicorrelated(3, rho) for _, _, rho in sc]
    structures = [{"kind": "equi", "rho": rho} for _, _, rho in sc]
    curves = [ScaleCurve(tab[s]["a"], tab[s]["scale"]) for s in range(n_scen)]
    for s in range(n_scen):
        if abs(tab[s]["rho"] - sc[s][2]) > 1e-15:
            raise RuntimeError("fwer_tables.json is stale for scenario %d" % s)
    qs = np.linspace(*Q_RANGE, g1)
    as_ = np.linspace(*A_RANGE, g2)
    return _grid_problem("c2", sigmas, structures, [(dp, dm) for dp, dm, _ in sc], curves,
                         qs, as_, 3, n_draws, keys)


def c3(n_scen=256, seed=0, draws_range=(1e5, 1e7)):
    """Batched uneven: d ~ U{3..10}, Sigma ~ LKJ(eta=2), 32..256 designs per
    scenario, mu_i ~ N(0.3, 0.2^2), Bonferroni thresholds, log-uniform N."""
    rng = np.random.default_rng(seed)
    sigmas, mus, bs, scen, nd = [], [], [], [], []
    lo, hi = math.log(draws_range[0]), math.log(draws_range[1])
    for s in range(n_scen):
        d = int(rng.integers(3, 11))
        sigmas.append(lkj_cvine(d, 2.0, rng))
        Js = int(rng.integers(32, 257))
        b = np.full(d, float(special.ndtri(1.0 - ALPHA0 / d)))
        for _ in range(Js):
            mus.append(rng.normal(0.3, 0.2, size=d))
            bs.append(b.copy())
            scen.append(s)
            nd.append(int(round(math.exp(rng.uniform(lo, hi)))))
    J = len(mus)
    return Problem("c3", sigmas, scen, mus, bs, nd, np.arange(J),
                   structures=[{"kind": "dense"}] * n_scen)


def c4(g1=32, g2=32, n_draws=10_000_000, keys="crn"):
    """d=10, AR(1) rho=0.3, 32 x 32 cutoff x allocation grid, delta = (0.5, 0.1)."""
    t = tables()["c4"]
    d, rho = 10, t["rho"]
    curve = ScaleCurve(t["a"], t["scale"])
    return _grid_problem("c4", [ar1(d, rho)], [{"kind": "ar1", "rho": rho}], [(0.5, 0.1)], [curve],
                         np.linspace(*Q_RANGE, g1), np.linspace(*A_RANGE, g2), d, n_draws, keys)


def c5(g1=64, g2=64, n_draws=10_000_000, keys="crn"):
    """d=20, 4 blocks of 5 (rho_in 0.6, rho_out 0.1), 64 x 64 grid, delta = (0.5, 0.1)."""
    t = tables()["c5"]
    sizes, rin, rout = t["sizes"], t["rho_in"], t["rho_out"]
    d = sum(sizes)
    curve = ScaleCurve(t["a"], t["scale"])
    return _grid_problem("c5", [block_equicorrelated(sizes, rin, rout)],
                         [{"kind": "block", "sizes": sizes, "rho_in": rin, "rho_out": rout}],
                         [(0.5, 0.1)], [curve], np.linspace(*Q_RANGE, g1), np.linspace(*A_RANGE, g2),
                         d, n_draws, keys)


def fwer_calibration(config="c2", n_draws=10_000_000, every=1, keys="crn"):
    """Designs for calibrating alpha splits to the FWER of Eq. 2 on the
    device: per scenario of `config` (c2: 16 equicorrelated d=3 scenarios;
    c4: AR(1) d=10; c5: block d=20) one design per allocation a on every
    `every`-th point of the stored table's grid, with split
    w(a) = (1 - a, a/(d-1), ...).  mu and b are placeholders (the
    calibration does not read them).  Returns (Problem, w packed [sum d],
    reference scales from the table, which the oracle wrote, allocations)."""
    t = tables()
    if config == "c2":
        scen = t["c2"]["scenarios"]
        sigmas = [equicorrelated(3, s["rho"]) for s in scen]
        structures = [{"kind": "equi", "rho": s["rho"]} for s in scen]
        grids = [(np.asarray(s["a"]), np.asarray(s["scale"])) for s in scen]
        d = 3
    elif config == "c4":
        c = t["c4"]
        d = c["d"]
        sigmas, structures = [ar1(d, c["rho"])], [{"kind": "ar1", "rho": c["rho"]}]
        grids = [(np.asarray(c["a"]), np.asarray(c["scale"]))]
    elif config == "c5":
        c = t["c5"]
        d = c["d"]
        sigmas = [block_equicorrelated(c["sizes"], c["rho_in"], c["rho_out"])]
        structures = [{"kind": "block", "sizes": c["sizes"], "rho_in": c["rho_in"], "rho_out": c["rho_out"]}]
        grids = [(np.asarray(c["a"]), np.asarray(c["scale"]))]
    else:
        raise ValueError(config)
    mus, bs, scen_of, ws, ref, alloc, key_list = [], [], [], [], [], [], []
    for s, (a_grid, s_grid) in enumerate(grids):
        for i in range(0, len(a_grid), every):
            ws.append(alloc_weights(float(a_grid[i]), d))
            ref.append(float(s_grid[i]))
            alloc.append(float(a_grid[i]))
            mus.append(np.zeros(d))
            bs.append(np.zeros(d))
            scen_of.append(s)
            key_list.append(s if keys == "crn" else len(mus) - 1)
    J = len(mus)
    prob = Problem("fwer-" + config, sigmas, scen_of, mus, bs, np.full(J, n_draws, np.uint64), key_list,
                   structures=structures)
    return prob, np.concatenate(ws), np.asarray(ref), np.asarray(alloc)


def c5_subsample(n=64, total=4096, seed=0):
    return np.sort(np.random.default_rng(seed).choice(total, n, replace=False))


def nested_sigma(r):
    """Correlation of the Z statistics of nested populations (Eq. 1):
    corr(X_k, X_l) = sqrt(r_l / r_k) for r_l <= r_k."""
    r = np.asarray(r, dtype=np.float64)
    lo, hi = np.minimum.outer(r, r), np.maximum.outer(r, r)
    return np.sqrt(lo / hi)


def paper_design(r, alpha, I3, delta0, prior_sd_scale=20.0):
    """Sampling law of one of the paper's designs with its Gaussian prior on
    the effect sizes (Eq. 1, 3, 10) folded in: X = X0 + S Delta with
    X0 ~ N(0, Sigma(r)), Delta ~ N(theta, Sigma_p), S = diag(sqrt(r_i I3)), so
    X ~ N(S theta, Sigma(r) + S Sigma_p S).  theta = -log(1 - Delta0),
    Sigma_p = Sigma(r) * (sigma sigma^T) with sigma_i = 1/sqrt(20 r_i), and the
    thresholds are b_i = Z_{1 - alpha_i}.  Returns (mean, covariance, b)."""
    r = np.asarray(r, dtype=np.float64)
    Sig = nested_sigma(r)
    theta = -np.log1p(-np.asarray(delta0, dtype=np.float64))
    sd = 1.0 / np.sqrt(prior_sd_scale * r)
    S = np.sqrt(r * I3)
    cov = Sig + np.outer(S, S) * Sig * np.outer(sd, sd)
    return S * theta, cov, special.ndtri(1.0 - np.asarray(alpha, dtype=np.float64))


def paper_optima(n_draws=10_000_000):
    """The optimal designs the paper reports for its biomarker conditions
    (Sec. 3): (a) no biomarker effect, (b) weak, (c) strong; one scenario
    each (the covariance depends on the design), keys 0, 1, 2."""
    cases = [([1.0], [0.025], 127.0, [0.25]),
             ([1.0, 0.365], [0.0163, 0.0107], 211.0, [0.3 - 0.1, 0.3 - 0.1 * 0.365]),
             ([1.0, 0.446, 0.168], [0.00194, 0.0135, 0.0133], 211.0,
              [0.8 - 0.6 * 1.0, 0.8 - 0.6 * 0.446, 0.8 - 0.6 * 0.168])]
    sig, mus, bs = [], [], []
    for r, alpha, I3v, d0 in cases:
        m, C, b = paper_design(r, alpha, I3v, d0)
        sig.append(C)
        mus.append(m)
        bs.append(b)
    return Problem("paper-optima", sig, [0, 1, 2], mus, bs, [n_draws] * 3, [0, 1, 2],
                   structures=[{"kind": "dense"}] * 3)


# The paper's reported optimal designs (Sec. 3): r, alpha, I3, hazard
# reductions Delta0 per population, for conditions (a) none, (b) weak and
# (c) strong biomarker effect.
PAPER_CONDITIONS = {
    "a": ([1.0], [0.025], 127.0, [0.25]),
    "b": ([1.0, 0.365], [0.0163, 0.0107], 211.0, [0.3 - 0.1, 0.3 - 0.1 * 0.365]),
    "c": ([1.0, 0.446, 0.168], [0.00194, 0.0135, 0.0133], 211.0,
          [0.8 - 0.6 * 1.0, 0.8 - 0.6 * 0.446, 0.8 - 0.6 * 0.168]),
}


def paper_two_layer_arrays(cond="c", N1=10240, N2=20480, alphas=None, seed=0, key=0, prior_sd_scale=20.0):
    """Packed inputs of the paper's two-layer estimator (Sec. 2.2, Eq. 5-7).

    Outer layer: N1 effect-size samples from the prior of Eq. 10 on the log
    hazard ratio, theta_k ~ N(theta_bar, Sigma_p) with theta_bar =
    -log(1 - Delta0) and Sigma_p = Sigma(r) * (sigma sigma^T), sigma_i =
    1/sqrt(20 r_i), drawn here with numpy default_rng(seed).  Inner layer: the
    engine's N2 draws x_l ~ N(0, Sigma(r)) (Eq. 1) of stream `key`, shared by
    every outer sample (the cross pairing of Eq. 7).  Design (a, k) tests the
    thresholds b_a = Z_{1 - alpha_a} against x + S theta_k, S = diag(sqrt(r I3)),
    i.e. mean shift mu = S theta_k.  `alphas` is a list of alpha vectors (the
    alpha points of one optimisation problem; default: the condition's
    reported optimum).  Designs are alpha-major: j = a N1 + k.
    Returns dict(sigma, mu[J, d], b[J, d], n_draws, key)."""
    r, alpha0, I3v, d0 = PAPER_CONDITIONS[cond]
    r = np.asarray(r, dtype=np.float64)
    d = r.shape[0]
    Sig = nested_sigma(r)
    theta_bar = -np.log1p(-np.asarray(d0, dtype=np.float64))
    sd = 1.0 / np.sqrt(prior_sd_scale * r)
    Lp = np.linalg.cholesky(Sig * np.outer(sd, sd))
    rng = np.random.default_rng(seed)
    theta = theta_bar + rng.standard_normal((N1, d)) @ Lp.T
    mu_k = theta * np.sqrt(r * I3v)
    A = np.atleast_2d(np.asarray(alpha0 if alphas is None else alphas, dtype=np.float64))
    b_a = special.ndtri(1.0 - A)
    mu = np.tile(mu_k, (A.shape[0], 1))
    b = np.repeat(b_a, N1, axis=0)
    return {"sigma": Sig, "mu": np.ascontiguousarray(mu), "b": np.ascontiguousarray(b), "n_draws": int(N2),
            "key": int(key), "cond": cond}


def paper_two_layer(cond="c", N1=1024, N2=4096, alphas=None, seed=0, key=0):
    """paper_two_layer_arrays as a Problem (one scenario, equal keys)."""
    a = paper_two_layer_arrays(cond, N1, N2, alphas, seed, key)
    J = a["mu"].shape[0]
    return Problem("paper-two-layer-" + cond, [a["sigma"]], np.zeros(J, np.int32), list(a["mu"]), list(a["b"]),
                   np.full(J, a["n_draws"], np.uint64), np.full(J, a["key"], np.uint64),
                   structures=[{"kind": "dense"}])


# Hazard reduction of the biomarker conditions as a function of the
# population fraction (Sec. 3): Delta_i = intercept + slope r_i, with I3.
PAPER_EFFECTS = {"a": (0.25, 0.0, 127.0), "b": (0.3, -0.1, 211.0), "c": (0.8, -0.6, 211.0)}


def paper_law(cond, r, prior_sd_scale=20.0):
    """Laws of condition `cond` at population fractions r (r_1 = 1): the
    Z statistics under the alternative with the prior folded in (mean,
    covariance; as in paper_design) and under the null, Sigma(r) (Eq. 1)."""
    icpt, slope, I3v = PAPER_EFFECTS[cond]
    r = np.asarray(r, dtype=np.float64)
    m, C, _ = paper_design(r, np.full(r.shape[0], 0.01), I3v, icpt + slope * r, prior_sd_scale)
    return m, C, nested_sigma(r)


def split_from_box(u):
    """Map points u of the box [0, 1]^(n-1) onto splits w of the alpha
    budget (the simplex of n weights): w_1 = u_1, w_j = u_j prod_{l<j}(1 - u_l),
    w_n = prod_l (1 - u_l).  Every split with FWER alpha0 is a ray of the
    constraint surface of Eq. 2, so the box covers the paper's design space
    of alpha with its constraint (the alpha scale is solved per split)."""
    u = np.atleast_2d(np.asarray(u, dtype=np.float64))
    rest = np.ones(u.shape[0])
    cols = []
    for j in range(u.shape[1]):
        cols.append(rest * u[:, j])
        rest = rest * (1.0 - u[:, j])
    cols.append(rest)
    return np.stack(cols, 1)


def box_points(n, k, seed=0):
    """n uniform points of [0, 1]^k (numpy default_rng(seed))."""
    return np.random.default_rng(seed).uniform(0.0, 1.0, (n, k))


def paper_r_pairs(step=0.05):
    """The paper's grid of nested populations for n = 3 (Sec. 3: 171 pairs):
    r = (1, r2, r3) with r2 > r3 on the grid step, 2 step, ..., 1 - step."""
    g = np.round(np.arange(step, 1.0 - step / 2, step), 10)
    return [(float(a), float(b)) for i, a in enumerate(g) for b in g[:i]]


def paper_alpha_points(cond="c", n=2000, seed=0, total=0.025):
    """n alpha vectors of a condition's dimension for timing one optimisation
    problem of the paper (N3 alpha points, Sec. 3): Dirichlet(1) weights
    scaled to sum `total` (a Bonferroni split of the FWER level)."""
    d = len(PAPER_CONDITIONS[cond][0])
    w = np.random.default_rng(seed).dirichlet(np.ones(d), size=n)
    return total * w


def design_at(config, q, a, scenario=0):
    """mu, b, dt/dtheta of one off-grid design of a grid config (for searches)."""
    if config == "c4":
        t = tables()["c4"]
        d, (dp, dm) = 10, (0.5, 0.1)
    elif config == "c5":
        t = tables()["c5"]
        d, (dp, dm) = 20, (0.5, 0.1)
    elif config == "c2":
        t = tables()["c2"]["scenarios"][scenario]
        dp, dm, _ = c2_scenarios(16)[scenario]
        d = 3
    else:
        raise ValueError(config)
    s, ds = ScaleCurve(t["a"], t["scale"])(a)
    return design_region(q, a, dp, dm, d, float(s), float(ds))


def random_problem(rng, n_scen=3, designs_per=(1, 6), d_choices=(1, 2, 3, 4, 5, 7, 10, 13, 20),
                   n_draws=(1, 5000), key_mode="independent"):
    """Small random problems (uneven d and N, ragged tails) for parity tests."""
    sigmas, mus, bs, scen, nd = [], [], [], [], []
    for s in range(n_scen):
        d = int(rng.choice(d_choices))
        sigmas.append(lkj_cvine(d, 2.0, rng) if d > 1 else np.eye(1))
        for _ in range(int(rng.integers(designs_per[0], designs_per[1] + 1))):
            mus.append(rng.normal(0.5, 0.7, size=d))
            b = rng.normal(1.5, 0.7, size=d)
            if d > 1 and rng.random() < 0.3:
                b[int(rng.integers(0, d))] = np.inf
            bs.append(b)
            scen.append(s)
            nd.append(int(rng.integers(n_draws[0], n_draws[1] + 1)))
    J = len(mus)
    keys = np.arange(J) if key_mode == "independent" else np.array(scen)
    begin = rng.integers(0, 1000, size=J)
    return Problem("random", sigmas, scen, mus, bs, nd, keys, draw_begin=begin,
                   structures=[{"kind": "dense"}] * n_scen)


def crn_groups(rng, d_list=(1, 3, 5, 8, 10, 13, 20), group=40, extra=3, n_draws=20_011, draw_begin=7,
               big_group_d=None, big_group=0):
    """Common-random-number groups for the shared-draw path: per dimension one
    LKJ(2) scenario with `group` designs sharing stream key, first draw and
    draw count, plus `extra` designs of their own keys; optionally one more
    group of `big_group` designs at dimension `big_group_d` (several chunks)."""
    sigmas, mus, bs, scen, nd, keys, begin = [], [], [], [], [], [], []
    specs = [(d, group) for d in d_list]
    if big_group_d is not None and big_group > 0:
        specs.append((big_group_d, big_group))
    key = 1000
    for s, (d, m) in enumerate(specs):
        sigmas.append(lkj_cvine(d, 2.0, rng) if d > 1 else np.eye(1))
        for k in range(m + extra):
            mus.append(rng.normal(0.5, 0.7, size=d))
            b = rng.normal(1.5, 0.7, size=d)
            if d > 1 and rng.random() < 0.2:
                b[int(rng.integers(0, d))] = np.inf
            bs.append(b)
            scen.append(s)
            nd.append(n_draws)
            begin.append(draw_begin)
            keys.append(s if k < m else key)
            key += 1
    return Problem("crn-groups", sigmas, scen, mus, bs, nd, keys, draw_begin=begin,
                   structures=[{"kind": "dense"}] * len(sigmas))
