"""Pins of the oracle's thin-plate spline (Sec. 2.3) against scipy's RBF
interpolator and the spline's defining properties."""
import numpy as np
import pytest

from oracle import tps

KERNELS = {1: "cubic", 2: "thin_plate_spline", 3: "linear"}


@pytest.mark.parametrize("k", [1, 2, 3])
@pytest.mark.parametrize("s", [0.0, 0.05, 1.0])
def test_matches_scipy_rbf(k, s):
    from scipy.interpolate import RBFInterpolator
    rng = np.random.default_rng(10 * k)
    x = rng.uniform(0, 1, (80, k))
    y = np.cos(2 * x).sum(1) + rng.normal(0, 0.05, 80)
    c, d = tps.fit(x, y, s)
    xq = rng.uniform(0, 1, (25, k))
    ref = RBFInterpolator(x, y, kernel=KERNELS[k], smoothing=s, degree=1)(xq)
    np.testing.assert_allclose(tps.evaluate(xq, x, c, d), ref, rtol=0, atol=1e-6 if s == 0 and k == 1 else 1e-9)


@pytest.mark.parametrize("k", [1, 2, 3])
def test_linear_data_are_reproduced(k):
    rng = np.random.default_rng(k)
    x = rng.uniform(-1, 1, (40, k))
    beta = rng.normal(size=k)
    y = 0.3 + x @ beta
    for s in (0.0, 0.7):
        c, d = tps.fit(x, y, s)
        np.testing.assert_allclose(c, 0.0, atol=1e-8)
        np.testing.assert_allclose(d, np.concatenate([[0.3], beta]), atol=1e-8)


def test_interpolation_and_fitted_identity():
    rng = np.random.default_rng(3)
    x = rng.uniform(0, 1, (50, 2))
    y = rng.normal(size=50)
    c, d = tps.fit(x, y, 0.0)
    np.testing.assert_allclose(tps.evaluate(x, x, c, d), y, atol=1e-9)
    s = 0.2
    c, d = tps.fit(x, y, s)
    np.testing.assert_allclose(tps.evaluate(x, x, c, d), y - s * c, atol=1e-10)
    # side conditions P^T c = 0
    np.testing.assert_allclose(np.hstack([np.ones((50, 1)), x]).T @ c, 0.0, atol=1e-10)


@pytest.mark.parametrize("k", [1, 2, 3])
def test_gradient_matches_differences(k):
    rng = np.random.default_rng(7 + k)
    x = rng.uniform(0, 1, (30, k))
    y = rng.normal(size=30)
    c, d = tps.fit(x, y, 0.1)
    z = rng.uniform(0.1, 0.9, k)
    h = 1e-6
    fd = np.array([(tps.evaluate(z + h * e, x, c, d)[0] - tps.evaluate(z - h * e, x, c, d)[0]) / (2 * h)
                   for e in np.eye(k)])
    np.testing.assert_allclose(tps.gradient(z, x, c, d), fd, rtol=1e-6, atol=1e-7)


def test_argmax_of_a_sampled_peak():
    # noise-free samples of a smooth peak: the fitted surface peaks where the
    # function does
    rng = np.random.default_rng(4)
    x = rng.uniform(0, 1, (400, 2))
    peak = np.array([0.62, 0.37])
    y = np.exp(-4.0 * ((x - peak) ** 2).sum(1))
    c, d = tps.fit(x, y, 0.0)
    xs, fs = tps.argmax(x, c, d, np.zeros(2), np.ones(2))
    np.testing.assert_allclose(xs, peak, atol=2e-3)
    assert fs == pytest.approx(1.0, abs=1e-3)


@pytest.mark.parametrize("k,s", [(1, 1e-3), (2, 0.01), (2, 0.3), (3, 0.05)])
def test_gcv_matches_the_influence_matrix(k, s):
    # V(s) = N |(I - A) y|^2 / tr(I - A)^2 with A built column by column from
    # fits to the unit vectors (A e_j = fitted values of the data e_j)
    rng = np.random.default_rng(40 + k)
    N = 40
    x = rng.uniform(0, 1, (N, k))
    y = np.sin(4 * x).sum(1) + rng.normal(0, 0.1, N)
    A = np.empty((N, N))
    for j in range(N):
        e = np.zeros(N)
        e[j] = 1.0
        c, d = tps.fit(x, e, s)
        A[:, j] = tps.evaluate(x, x, c, d)
    r = y - A @ y
    ref = N * (r @ r) / np.trace(np.eye(N) - A) ** 2
    assert tps.gcv(x, y, s) == pytest.approx(ref, rel=1e-8)


def test_gcv_prefers_smoothing_noisy_data():
    rng = np.random.default_rng(8)
    x = rng.uniform(0, 1, (120, 2))
    y = np.exp(-3 * ((x - 0.5) ** 2).sum(1)) + rng.normal(0, 0.05, 120)
    grid = np.logspace(-8, 1, 19)
    scores = [tps.gcv(x, y, s) for s in grid]
    best = grid[int(np.argmin(scores))]
    assert 1e-6 < best < 10.0        # neither interpolation nor the plane
    assert min(scores) < scores[0] and min(scores) < scores[-1]
