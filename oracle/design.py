"""Design model and objective as functions of the design parameters (oracle).

TEST INFRASTRUCTURE ONLY: imported by tests and by the threshold-table
script, never by the CUDA library.

An independent restatement of how a design becomes a rejection region, so
that tests can check the input module against it and take finite
differences of the exact objective.

Model (Sec. 2.1, Eq. 3 and Sec. 3, Eq. 9-10; readings of the benchmark's
cutoff / allocation parametrisation):
  * cutoff quantile q in (0,1) of a N(0,1) biomarker; the d nested populations
    hold the fractions r_i = 1 - q (i-1)/(d-1), so r_1 = 1 (whole population)
    and r_d = 1 - q (patients above the cutoff);
  * hazard reduction linear in r (the family of Sec. 3 conditions (b), (c)):
    Delta_i = delta_plus - (delta_plus - delta_minus) r_i;
  * log hazard ratio theta_i = -log(1 - Delta_i) (Sec. 3, below Eq. 10);
  * mean of the Z statistics mu_i = sqrt(r_i I3) theta_i (Eq. 3);
  * alpha allocation: weights w = (1 - a, a/(d-1), ..., a/(d-1)), alpha = s w,
    the scale s solving the FWER constraint 1 - Phi_Sigma(b) = alpha_0 (Eq. 2),
    b_i = Z_{1 - alpha_i}.
"""
import math

import numpy as np

from . import quad


def information_units(alpha=0.025, beta=0.1, delta=0.2):
    """I3 = (Z_{1-alpha} + Z_{1-beta})^2 / log(1 - Delta)^2 (Sec. 3, Eq. 9)."""
    z = quad.norm_ppf(1.0 - alpha) + quad.norm_ppf(1.0 - beta)
    return float(z * z / math.log(1.0 - delta) ** 2)


def fractions(q, d):
    i = np.arange(d, dtype=np.float64)
    return 1.0 - q * i / (d - 1) if d > 1 else np.ones(1)


def mean_shift(q, delta_plus, delta_minus, d, I3):
    r = fractions(q, d)
    Delta = delta_plus - (delta_plus - delta_minus) * r
    theta = -np.log1p(-Delta)
    return np.sqrt(r * I3) * theta


def alloc_weights(a, d):
    w = np.full(d, a / (d - 1))
    w[0] = 1.0 - a
    return w


def objective(q, a, delta_plus, delta_minus, d, I3, alpha0, Sigma=None, structure=None,
              scale_cache=None):
    """P(success) of one design by quadrature: 1 - Phi_Sigma(b(a) - mu(q, delta))."""
    w = alloc_weights(a, d)
    key = (round(a, 15),)
    if scale_cache is not None and key in scale_cache:
        s = scale_cache[key]
    else:
        s = quad.calibrate_scale(w, alpha0, Sigma, structure)
        if scale_cache is not None:
            scale_cache[key] = s
    b = quad.thresholds(s, w)
    mu = mean_shift(q, delta_plus, delta_minus, d, I3)
    return quad.success_probability(mu, b, Sigma, structure)


def objective_fd_gradient(theta, d, I3, alpha0, Sigma=None, structure=None, step=1e-4):
    """Central differences of the exact objective in theta = (q, a, d+, d-)."""
    theta = np.asarray(theta, dtype=np.float64)
    g = np.zeros(4)
    for k in range(4):
        e = np.zeros(4)
        e[k] = step
        hi = objective(*(theta + e), d, I3, alpha0, Sigma, structure)
        lo = objective(*(theta - e), d, I3, alpha0, Sigma, structure)
        g[k] = (hi - lo) / (2 * step)
    return g


def collapsed_prior(r, I3, Delta0, prior_sd_scale=80.0 / 4.0):
    """Gaussian prior of Eq. 10 folded into the sampling distribution.

    With Delta ~ N(theta, Sigma_p) independent of X0 ~ N(0, Sigma(r)) (Eq. 1),
    X = X0 + S Delta with S = diag(sqrt(r_i I3)) is N(S theta, Sigma(r) + S Sigma_p S),
    so the expected power (Eq. 4) is one orthant probability of that law.
    Returns (mean, covariance) for the populations with r_i > 0.
    """
    r = np.asarray(r, dtype=np.float64)
    d = r.shape[0]
    Sig = np.empty((d, d))
    for k in range(d):
        for l in range(d):
            lo, hi = min(r[k], r[l]), max(r[k], r[l])
            Sig[k, l] = math.sqrt(lo / hi)
    theta = -np.log1p(-np.asarray(Delta0, dtype=np.float64))
    sd = 1.0 / np.sqrt(prior_sd_scale * r)
    Sp = Sig * np.outer(sd, sd)
    S = np.sqrt(r * I3)
    return S * theta, Sig + np.outer(S, S) * Sp


def two_layer_moments(r, alpha, I3, Delta0, prior_sd_scale=80.0 / 4.0):
    """Moments of the indicator of the paper's two-layer estimator (Sec. 2.2).

    Eq. 5-7 average h(theta_k, x_l) = 1{some x_l,i + S_i theta_k,i > b_i} over
    all pairs of N1 outer samples theta_k ~ N(theta_bar, Sigma_p) (the prior
    of Eq. 10 on the log hazard ratio) and N2 inner samples x_l ~ N(0, Sigma(r))
    (Eq. 1), with S = diag(sqrt(r_i I3)) and b_i = Z_{1 - alpha_i}.
    Returns (P, s2, s_theta2, s_x2):
      P        = E h = 1 - Phi_C(b - S theta_bar),  C = Sigma + S Sigma_p S;
      s2       = Var h = P (1 - P);
      s_theta2 = Var_theta E_x h  (two draws sharing theta: Cov = S Sigma_p S);
      s_x2     = Var_x E_theta h  (two draws sharing x:     Cov = Sigma).
    E[h h'] for a shared component is 1 - 2 (1 - P) + Phi_6(b - m, b - m) of
    the stacked 2d-vector; the 2d-dimensional normal CDF is scipy's (Genz)
    routine, the d-dimensional orthant the quadrature of quad.orthant.
    """
    from scipy.stats import multivariate_normal
    r = np.asarray(r, dtype=np.float64)
    d = r.shape[0]
    Sig = np.empty((d, d))
    for k in range(d):
        for l in range(d):
            lo, hi = min(r[k], r[l]), max(r[k], r[l])
            Sig[k, l] = math.sqrt(lo / hi)
    theta = -np.log1p(-np.asarray(Delta0, dtype=np.float64))
    sd = 1.0 / np.sqrt(prior_sd_scale * r)
    S = np.sqrt(r * I3)
    SSpS = np.outer(S, S) * Sig * np.outer(sd, sd)
    C = Sig + SSpS
    t = quad.norm_ppf(1.0 - np.asarray(alpha, dtype=np.float64)) - S * theta
    F = quad.orthant(t, C)
    P = 1.0 - F

    def both(cross):
        big = np.block([[C, cross], [cross.T, C]])
        kw = dict(mean=np.zeros(2 * d), cov=big, abseps=1e-7, releps=1e-7, maxpts=2_000_000 * d)
        try:
            F2 = multivariate_normal.cdf(np.concatenate([t, t]), rng=np.random.default_rng(0), **kw)
        except TypeError:                                   # scipy without the rng keyword
            F2 = multivariate_normal.cdf(np.concatenate([t, t]), **kw)
        return 1.0 - 2.0 * F + F2

    return P, P * (1.0 - P), both(SSpS) - P * P, both(Sig) - P * P


def two_layer_variance(N1, N2, moments):
    """Exact variance of the Eq. 7 estimator (a two-sample U-statistic): pairs
    that share theta_k covary by s_theta2, pairs that share x_l by s_x2, so
    Var = [s2 + (N2 - 1) s_theta2 + (N1 - 1) s_x2] / (N1 N2).  Appendix A.2's
    bound 1/(4 N1 N2) covers only the first term."""
    _, s2, sth, sx = moments
    return (s2 + (N2 - 1) * sth + (N1 - 1) * sx) / (N1 * N2)
