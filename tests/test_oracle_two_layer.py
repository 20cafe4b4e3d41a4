"""Pins of the oracle's variance of the paper's two-layer estimator (Sec. 2.2,
Eq. 5-8, Appendix A.2) by brute-force simulation on the CPU."""
import numpy as np
import pytest

import workloads
from oracle import design, quad


@pytest.fixture(scope="module")
def strong():
    r, alpha, I3, d0 = workloads.PAPER_CONDITIONS["c"]
    return (r, alpha, I3, d0), design.two_layer_moments(r, alpha, I3, d0)


def simulate(cond, N1, N2, reps, seed):
    """Eq. 7 repeated `reps` times with plain numpy draws: outer theta from the
    prior of Eq. 10, inner x from N(0, Sigma(r)) of Eq. 1, every pair tested."""
    r, alpha, I3, d0 = cond
    r = np.asarray(r, dtype=np.float64)
    d = r.shape[0]
    Sig = np.sqrt(np.minimum.outer(r, r) / np.maximum.outer(r, r))
    sd = 1.0 / np.sqrt(20.0 * r)
    rng = np.random.default_rng(seed)
    theta = -np.log1p(-np.asarray(d0)) + rng.multivariate_normal(np.zeros(d), Sig * np.outer(sd, sd), (reps, N1))
    x = rng.multivariate_normal(np.zeros(d), Sig, (reps, N2))
    b = quad.norm_ppf(1.0 - np.asarray(alpha))
    y = x[:, None, :, :] + (theta * np.sqrt(r * I3))[:, :, None, :]      # (reps, N1, N2, d)
    return np.any(y > b, axis=-1).mean(axis=(1, 2))


@pytest.mark.parametrize("N1,N2,reps", [(1, 1, 400_000), (4, 8, 200_000), (16, 1, 200_000), (1, 16, 200_000)])
def test_two_layer_variance_matches_simulation(strong, N1, N2, reps):
    cond, m = strong
    est = simulate(cond, N1, N2, reps, seed=N1 * 100 + N2)
    V = design.two_layer_variance(N1, N2, m)
    assert abs(est.mean() - m[0]) <= 5 * np.sqrt(V / reps)
    assert est.var(ddof=1) == pytest.approx(V, rel=0.06)


def test_one_pair_is_a_bernoulli(strong):
    _, m = strong
    P, s2, _, _ = m
    assert P == pytest.approx(0.97699, abs=1e-4)          # the strong-biomarker optimum, Sec. 3 (0.977)
    assert design.two_layer_variance(1, 1, m) == pytest.approx(s2, rel=1e-12)
    assert s2 == pytest.approx(P * (1 - P), rel=1e-12)


def test_appendix_bound_misses_the_shared_sample_terms(strong):
    # Eq. 8 bounds Var(P_hat) by 1/(4 N1 N2) = 1.19e-9 at N1 = 10240,
    # N2 = 20480; with one inner sample set shared by all outer samples the
    # variance is about 1e3 times larger (the outer-layer term s_theta2 / N1).
    _, m = strong
    N1, N2 = 10240, 20480
    V = design.two_layer_variance(N1, N2, m)
    assert 1.0 / (4 * N1 * N2) == pytest.approx(1.19e-9, rel=2e-3)
    assert V > 500 * (1.0 / (4 * N1 * N2))
    assert V == pytest.approx(m[2] / N1, rel=0.05)
