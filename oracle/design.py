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
