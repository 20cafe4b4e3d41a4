"""Deterministic FP64 values of the design objective (oracle, test infrastructure).

TEST INFRASTRUCTURE ONLY: used by tests, by the CPU-baseline leg of the
benchmark and by the script that writes the threshold tables.  Nothing in
the CUDA library imports this module.

The objective of Sec. 2.1 (Eq. 4 with a point prior, and Eq. 2 at mu = 0) is
an orthant probability of a correlated normal vector:

    P(success) = 1 - Phi_Sigma(b - mu),   Phi_Sigma(t) = P(Y <= t), Y ~ N(0, Sigma).

This module evaluates Phi_Sigma by deterministic quadrature:

* ``orthant_dense``  -- any Sigma with d <= 3, by sequential conditioning on
  the Cholesky factor (the textbook Genz transformation), nested composite
  Gauss-Legendre refined until two successive refinements agree.
* ``orthant_equi``   -- equicorrelated Sigma (rho >= 0), any d, through the
  one-factor representation Y_i = sqrt(rho) U + sqrt(1 - rho) E_i.
* ``orthant_ar1``    -- AR(1) Sigma_ij = rho^|i-j|, any d, by the Markov
  recursion of the chain Y_{i+1} = rho Y_i + sqrt(1 - rho^2) E_{i+1}.
* ``orthant_block``  -- block-equicorrelated Sigma (rho_in within a block,
  rho_out across, 0 <= rho_out <= rho_in), any d, through the two-level
  factor representation.

Each routine truncates the real line at +-TRUNC (normal tail 1e-33) and
refines the rule until successive values differ by less than ``tol``.
A threshold of +inf drops that coordinate (alpha_i = 0 in Eq. 2).
"""
import math

import numpy as np
from scipy import optimize, special

TRUNC = 12.0
SQRT2 = math.sqrt(2.0)
INV_SQRT_2PI = 1.0 / math.sqrt(2.0 * math.pi)


def norm_cdf(x):
    """Standard normal CDF, 0.5 * erfc(-x / sqrt 2)."""
    return 0.5 * special.erfc(-np.asarray(x, dtype=np.float64) / SQRT2)


def norm_pdf(x):
    x = np.asarray(x, dtype=np.float64)
    return INV_SQRT_2PI * np.exp(-0.5 * x * x)


def norm_ppf(p):
    """Standard normal quantile (Z_p in the paper's notation)."""
    return special.ndtri(p)


_GL_CACHE = {}


def _gauss_legendre(m):
    if m not in _GL_CACHE:
        _GL_CACHE[m] = np.polynomial.legendre.leggauss(m)
    return _GL_CACHE[m]


def composite_rule(lo, hi, panels, m=20):
    """Nodes and weights of a composite m-point Gauss-Legendre rule.

    lo, hi: arrays of equal shape (S,) -> nodes, weights of shape (S, panels*m).
    Intervals with hi <= lo get zero weight.
    """
    lo = np.atleast_1d(np.asarray(lo, dtype=np.float64))
    hi = np.atleast_1d(np.asarray(hi, dtype=np.float64))
    hi = np.maximum(hi, lo)
    x, w = _gauss_legendre(m)
    frac = np.linspace(0.0, 1.0, panels + 1)
    edges = lo[:, None] + (hi - lo)[:, None] * frac[None, :]
    a, b = edges[:, :-1], edges[:, 1:]
    half = 0.5 * (b - a)
    mid = 0.5 * (a + b)
    nodes = mid[:, :, None] + half[:, :, None] * x[None, None, :]
    weights = half[:, :, None] * w[None, None, :]
    S = lo.shape[0]
    return nodes.reshape(S, -1), weights.reshape(S, -1)


def _refine(fn, tol, start=4, max_panels=1024):
    """Evaluate fn(panels) with doubling panel counts until converged."""
    panels = start
    prev = fn(panels)
    while True:
        panels *= 2
        cur = fn(panels)
        if abs(cur - prev) <= tol or panels >= max_panels:
            if abs(cur - prev) > max(tol, 1e-9):
                raise RuntimeError("quadrature did not converge: %r vs %r" % (prev, cur))
            return cur
        prev = cur


# ---------------------------------------------------------------- dense d<=3
def orthant_dense(t, Sigma, tol=1e-13):
    """P(Y <= t) for Y ~ N(0, Sigma), d = len(t) <= 3, by conditioning.

    With Sigma = L L^T and Y = L Z:
      d=1: Phi(t1 / L11)
      d=2: int_{z1 < t1/L11} phi(z1) Phi((t2 - L21 z1) / L22) dz1
      d=3: int_{z1 < t1/L11} phi(z1) int_{z2 < (t2 - L21 z1)/L22} phi(z2)
               Phi((t3 - L31 z1 - L32 z2) / L33) dz2 dz1
    """
    t = np.asarray(t, dtype=np.float64)
    Sigma = np.asarray(Sigma, dtype=np.float64)
    d = t.shape[0]
    if d == 0:
        return 1.0
    if d > 3:
        raise ValueError("orthant_dense handles d <= 3")
    L = np.linalg.cholesky(Sigma)
    if d == 1:
        return float(norm_cdf(t[0] / L[0, 0]))

    def upper(val):
        return np.where(np.isposinf(val), TRUNC, np.minimum(val, TRUNC))

    if d == 2:
        def fn(panels):
            u1 = upper(np.array([t[0] / L[0, 0]]))
            z1, w1 = composite_rule([-TRUNC], u1, panels)
            inner = norm_cdf((t[1] - L[1, 0] * z1) / L[1, 1])
            return float(np.sum(w1 * norm_pdf(z1) * inner))
        return _refine(fn, tol)

    def fn3(panels):
        u1 = upper(np.array([t[0] / L[0, 0]]))
        z1, w1 = composite_rule([-TRUNC], u1, panels)
        z1, w1 = z1[0], w1[0]
        u2 = upper((t[1] - L[1, 0] * z1) / L[1, 1])
        z2, w2 = composite_rule(np.full_like(z1, -TRUNC), u2, panels)
        inner = norm_cdf((t[2] - L[2, 0] * z1[:, None] - L[2, 1] * z2) / L[2, 2])
        f2 = np.sum(w2 * norm_pdf(z2) * inner, axis=1)
        return float(np.sum(w1 * norm_pdf(z1) * f2))
    return _refine(fn3, tol)


# ------------------------------------------------------------ equicorrelated
def orthant_equi(t, rho, tol=1e-13):
    """P(Y <= t), Sigma = (1-rho) I + rho 11^T with 0 <= rho < 1:
    int phi(u) prod_i Phi((t_i - sqrt(rho) u) / sqrt(1 - rho)) du."""
    t = np.asarray(t, dtype=np.float64)
    if not (0.0 <= rho < 1.0):
        raise ValueError("orthant_equi needs 0 <= rho < 1")
    if rho == 0.0:
        return float(np.prod(norm_cdf(t)))
    a, c = math.sqrt(rho), math.sqrt(1.0 - rho)

    def fn(panels):
        u, w = composite_rule([-TRUNC], [TRUNC], panels)
        u, w = u[0], w[0]
        vals = norm_cdf((t[None, :] - a * u[:, None]) / c)
        return float(np.sum(w * norm_pdf(u) * np.prod(vals, axis=1)))
    return _refine(fn, tol)


# --------------------------------------------------------------------- AR(1)
def orthant_ar1(t, rho, tol=1e-13):
    """P(Y <= t), Sigma_ij = rho^|i-j|, |rho| < 1, by the Markov recursion
    g_1(x) = phi(x);  g_{i+1}(x') = int_{x <= t_i} g_i(x) phi((x' - rho x)/s)/s dx,
    s = sqrt(1 - rho^2);  P = int_{x <= t_d} g_d(x) dx."""
    t = np.asarray(t, dtype=np.float64)
    d = t.shape[0]
    s = math.sqrt(1.0 - rho * rho)
    up = np.where(np.isposinf(t), TRUNC, np.minimum(t, TRUNC))

    def fn(panels):
        x, w = composite_rule([-TRUNC], [up[0]], panels)
        x, w = x[0], w[0]
        g = norm_pdf(x)
        for i in range(1, d):
            xn, wn = composite_rule([-TRUNC], [up[i]], panels)
            xn, wn = xn[0], wn[0]
            K = norm_pdf((xn[:, None] - rho * x[None, :]) / s) / s
            g = K @ (w * g)
            x, w = xn, wn
        return float(np.sum(w * g))
    return _refine(fn, tol, start=8)


# -------------------------------------------------------- block-equicorrelated
def orthant_block(t, sizes, rho_in, rho_out, tol=1e-12):
    """P(Y <= t) for unit-variance Y with corr rho_in inside a block and rho_out
    across blocks (0 <= rho_out <= rho_in < 1):
      Y_i = sqrt(rho_out) G + sqrt(rho_in - rho_out) B_k + sqrt(1 - rho_in) E_i,
      P = int phi(g) prod_k [ int phi(u) prod_{i in k} Phi((t_i - sqrt(rho_out) g
            - sqrt(rho_in - rho_out) u) / sqrt(1 - rho_in)) du ] dg."""
    t = np.asarray(t, dtype=np.float64)
    if not (0.0 <= rho_out <= rho_in < 1.0):
        raise ValueError("orthant_block needs 0 <= rho_out <= rho_in < 1")
    if sum(sizes) != t.shape[0]:
        raise ValueError("block sizes do not add up to d")
    ag, au, ae = math.sqrt(rho_out), math.sqrt(rho_in - rho_out), math.sqrt(1.0 - rho_in)
    starts = np.cumsum([0] + list(sizes))

    def fn(panels):
        g, wg = composite_rule([-TRUNC], [TRUNC], panels)
        g, wg = g[0], wg[0]
        u, wu = composite_rule([-TRUNC], [TRUNC], panels)
        u, wu = u[0], wu[0]
        total = wg * norm_pdf(g)
        for k in range(len(sizes)):
            tk = t[starts[k]:starts[k + 1]]
            arg = (tk[None, None, :] - ag * g[:, None, None] - au * u[None, :, None]) / ae
            inner = np.prod(norm_cdf(arg), axis=2)
            total = total * np.sum(wu * norm_pdf(u) * inner, axis=1)
        return float(np.sum(total))
    return _refine(fn, tol, start=8, max_panels=256)


# ------------------------------------------------------------------ dispatch
def orthant(t, Sigma=None, structure=None, tol=None):
    """Phi_Sigma(t) by the routine matching ``structure``.

    structure: None / {"kind": "dense"} (d <= 3), {"kind": "equi", "rho"},
    {"kind": "ar1", "rho"}, {"kind": "block", "sizes", "rho_in", "rho_out"},
    {"kind": "diag"}.  When Sigma is also given it must match the structure.
    """
    t = np.asarray(t, dtype=np.float64)
    kind = (structure or {"kind": "dense"})["kind"]
    if Sigma is not None and structure is not None and kind != "dense":
        ref = structured_sigma(t.shape[0], structure)
        if not np.allclose(ref, Sigma, atol=1e-14, rtol=0):
            raise ValueError("Sigma does not match its stated structure")
    kw = {} if tol is None else {"tol": tol}
    if kind == "dense":
        return orthant_dense(t, Sigma, **kw)
    if kind == "diag":
        return float(np.prod(norm_cdf(t)))
    if kind == "equi":
        return orthant_equi(t, structure["rho"], **kw)
    if kind == "ar1":
        return orthant_ar1(t, structure["rho"], **kw)
    if kind == "block":
        return orthant_block(t, structure["sizes"], structure["rho_in"], structure["rho_out"], **kw)
    raise ValueError("unknown structure %r" % kind)


def structured_sigma(d, structure):
    """The correlation matrix that a structure descriptor stands for."""
    kind = structure["kind"]
    if kind == "diag":
        return np.eye(d)
    if kind == "equi":
        r = structure["rho"]
        return (1.0 - r) * np.eye(d) + r * np.ones((d, d))
    if kind == "ar1":
        idx = np.arange(d)
        return structure["rho"] ** np.abs(idx[:, None] - idx[None, :])
    if kind == "block":
        S = np.full((d, d), structure["rho_out"])
        start = 0
        for n in structure["sizes"]:
            S[start:start + n, start:start + n] = structure["rho_in"]
            start += n
        np.fill_diagonal(S, 1.0)
        return S
    raise ValueError("no fixed matrix for structure %r" % kind)


def success_probability(mu, b, Sigma=None, structure=None):
    """P(X_i > b_i for some i), X ~ N(mu, Sigma): 1 - Phi_Sigma(b - mu) (Eq. 4)."""
    t = np.asarray(b, dtype=np.float64) - np.asarray(mu, dtype=np.float64)
    return 1.0 - orthant(t, Sigma, structure)


# -------------------------------------------------------- FWER calibration
def fwer(b, Sigma=None, structure=None):
    """Family-wise error rate 1 - Phi_Sigma(b) under H0 (Eq. 2)."""
    return 1.0 - orthant(np.asarray(b, dtype=np.float64), Sigma, structure)


def thresholds(scale, weights):
    """b_i = Z_{1 - alpha_i}, alpha_i = scale * w_i; w_i = 0 gives +inf."""
    w = np.asarray(weights, dtype=np.float64)
    alpha = scale * w
    with np.errstate(divide="ignore"):
        return np.where(w > 0, norm_ppf(1.0 - alpha), np.inf)


def calibrate_scale(weights, alpha0, Sigma=None, structure=None, xtol=1e-15):
    """Solve 1 - Phi_Sigma(b(s)) = alpha0 for the scale s of alpha = s * w (Eq. 2).

    FWER(s) increases in s; it lies between max_i alpha_i and sum_i alpha_i
    (Bonferroni), which brackets the root in [alpha0 / sum w, alpha0 / max w].
    """
    w = np.asarray(weights, dtype=np.float64)
    lo, hi = alpha0 / w.sum(), alpha0 / w.max()
    if hi - lo <= 1e-300:
        return lo

    def g(s):
        return fwer(thresholds(s, w), Sigma, structure) - alpha0
    glo, ghi = g(lo), g(hi)
    if glo > 0 or ghi < 0:
        # The bracket ends are exact solutions up to quadrature error.
        return lo if abs(glo) < abs(ghi) else hi
    return optimize.brentq(g, lo, hi, xtol=xtol, rtol=4 * np.finfo(float).eps, maxiter=200)
