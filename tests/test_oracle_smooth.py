"""Pins of the oracle's local-polynomial smoother and argmax (Sec. 2.3)."""
import numpy as np
import pytest

from oracle import smooth


def test_reproduces_quadratics_exactly():
    # a degree-2 local fit reproduces any quadratic surface, edges included
    G1, G2 = 9, 11
    i, j = np.meshgrid(np.arange(G1), np.arange(G2), indexing="ij")
    P = 0.3 + 0.01 * i - 0.02 * j + 0.003 * i * i - 0.001 * i * j + 0.002 * j * j
    np.testing.assert_allclose(smooth.smooth_grid(P), P, rtol=0, atol=1e-13)
    x = np.arange(15.0)
    P1 = (0.5 - 0.01 * x + 0.002 * x * x)[None, :]
    np.testing.assert_allclose(smooth.smooth_grid(P1), P1, rtol=0, atol=1e-13)
    np.testing.assert_allclose(smooth.smooth_grid(P1.T), P1.T, rtol=0, atol=1e-13)


def test_degree_zero_is_weighted_mean():
    P = np.random.default_rng(0).random((7, 7))
    S = smooth.smooth_grid(P, bandwidth=3.0, degree=0)
    w = smooth.tricube(np.arange(-2, 3) / 3.0)
    W = np.outer(w, w)
    assert S[3, 3] == pytest.approx(np.sum(W * P[1:6, 1:6]) / W.sum(), abs=1e-14)


def test_interior_equivalent_kernel_is_symmetric():
    # at an interior point the smoother is a fixed linear stencil that sums to 1
    # and is symmetric under reflections of the grid
    G = 9
    stencil = np.zeros((5, 5))
    for a in range(5):
        for b in range(5):
            E = np.zeros((G, G))
            E[2 + a, 2 + b] = 1.0
            stencil[a, b] = smooth.smooth_grid(E)[4, 4]
    assert stencil.sum() == pytest.approx(1.0, abs=1e-13)
    np.testing.assert_allclose(stencil, stencil[::-1, :], atol=1e-14)
    np.testing.assert_allclose(stencil, stencil.T, atol=1e-14)


def test_noise_reduction():
    rng = np.random.default_rng(1)
    i, j = np.meshgrid(np.arange(32), np.arange(32), indexing="ij")
    truth = 0.8 - 0.0005 * (i - 20) ** 2 - 0.0003 * (j - 12) ** 2
    noisy = truth + rng.normal(0, 0.01, truth.shape)
    err_raw = np.abs(noisy - truth).mean()
    err_sm = np.abs(smooth.smooth_grid(noisy) - truth).mean()
    assert err_sm < 0.6 * err_raw


def test_argmax_lowest_index_on_ties():
    v = np.array([[0.1, 0.5, 0.2], [0.5, 0.3, 0.5]])
    assert smooth.argmax_lowest(v) == (1, 0.5)
    sm, idx, val, ridx, rval = smooth.smooth_argmax(np.stack([v, v[::-1]]), 2, 3, bandwidth=1.5, degree=0)
    assert ridx[0] == 1 and ridx[1] == 0
