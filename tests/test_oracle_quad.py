"""Pins of the oracle's deterministic orthant probabilities (Eq. 2, Eq. 4)
against closed forms, special cases and an independent library routine."""
import json
import math
import os

import numpy as np
import pytest
from scipy.stats import multivariate_normal

from oracle import design, quad

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def rand_corr(d, rng):
    A = rng.normal(size=(d, d))
    S = A @ A.T + 0.3 * np.eye(d)
    D = np.sqrt(np.diag(S))
    return S / np.outer(D, D)


def test_d1_closed_form():
    for t in [-3.0, -0.4, 0.0, 1.2, 4.0]:
        assert quad.orthant_dense(np.array([t]), np.eye(1)) == pytest.approx(0.5 * math.erfc(-t / math.sqrt(2)), abs=1e-15)


def test_bivariate_orthant_identity():
    # P(Y1 <= 0, Y2 <= 0) = 1/4 + arcsin(rho) / (2 pi)   (Sheppard)
    for rho in [-0.9, -0.3, 0.0, 0.45, 0.8, 0.97]:
        S = np.array([[1.0, rho], [rho, 1.0]])
        assert quad.orthant_dense(np.zeros(2), S) == pytest.approx(0.25 + math.asin(rho) / (2 * math.pi), abs=1e-12)


def test_trivariate_orthant_identity():
    # P(Y <= 0) = 1/8 + (asin r12 + asin r13 + asin r23) / (4 pi)
    rng = np.random.default_rng(0)
    for _ in range(5):
        R = rand_corr(3, rng)
        ref = 0.125 + (math.asin(R[0, 1]) + math.asin(R[0, 2]) + math.asin(R[1, 2])) / (4 * math.pi)
        assert quad.orthant_dense(np.zeros(3), R) == pytest.approx(ref, abs=1e-12)
    R = quad.structured_sigma(3, {"kind": "equi", "rho": 0.5})
    assert quad.orthant_dense(np.zeros(3), R) == pytest.approx(0.25, abs=1e-13)


def test_diagonal_product():
    rng = np.random.default_rng(1)
    for d in [1, 2, 3]:
        t = rng.normal(size=d)
        D = np.diag(rng.uniform(0.5, 2.0, size=d))
        ref = np.prod(quad.norm_cdf(t / np.sqrt(np.diag(D))))
        assert quad.orthant_dense(t, D) == pytest.approx(ref, abs=1e-13)


def test_against_library_genz():
    rng = np.random.default_rng(3)
    for d in [2, 3]:
        for _ in range(4):
            R = rand_corr(d, rng)
            t = rng.normal(0.5, 1.0, size=d)
            lib = multivariate_normal.cdf(t, cov=R, abseps=1e-12, releps=1e-12, maxpts=10**7)
            assert quad.orthant_dense(t, R) == pytest.approx(lib, abs=2e-8)


def test_infinite_threshold_drops_coordinate():
    rng = np.random.default_rng(4)
    R = rand_corr(3, rng)
    t = np.array([0.3, np.inf, -0.2])
    sub = R[np.ix_([0, 2], [0, 2])]
    assert quad.orthant_dense(t, R) == pytest.approx(quad.orthant_dense(t[[0, 2]], sub), abs=1e-13)


def test_structured_routines_agree_with_dense_at_d3():
    rng = np.random.default_rng(5)
    for _ in range(3):
        t = rng.normal(0.8, 1.0, size=3)
        for st in [{"kind": "equi", "rho": 0.35}, {"kind": "ar1", "rho": 0.6},
                   {"kind": "ar1", "rho": -0.4}, {"kind": "block", "sizes": [2, 1], "rho_in": 0.7, "rho_out": 0.2}]:
            S = quad.structured_sigma(3, st)
            assert quad.orthant(t, S, st) == pytest.approx(quad.orthant_dense(t, S), abs=1e-12)


def test_block_reduces_to_equicorrelated():
    t = np.linspace(0.5, 2.5, 12)
    a = quad.orthant_block(t, [4, 4, 4], 0.4, 0.4)
    b = quad.orthant_equi(t, 0.4)
    assert a == pytest.approx(b, abs=1e-12)


def test_ar1_zero_correlation_is_product():
    t = np.linspace(-0.5, 2.0, 10)
    assert quad.orthant_ar1(t, 0.0) == pytest.approx(float(np.prod(quad.norm_cdf(t))), abs=1e-13)


def test_high_dimension_against_library_qmc():
    # scipy's randomised lattice rule (Genz-Bretz) is accurate to ~1e-6 here
    t = np.full(10, 2.6)
    S = quad.structured_sigma(10, {"kind": "ar1", "rho": 0.3})
    lib = multivariate_normal.cdf(t, cov=S, maxpts=2_000_000, abseps=1e-9, rng=np.random.default_rng(0))
    assert quad.orthant_ar1(t, 0.3) == pytest.approx(lib, abs=3e-6)
    t = np.linspace(2.0, 3.5, 20)
    st = {"kind": "block", "sizes": [5, 5, 5, 5], "rho_in": 0.6, "rho_out": 0.1}
    S = quad.structured_sigma(20, st)
    lib = multivariate_normal.cdf(t, cov=S, maxpts=2_000_000, abseps=1e-9, rng=np.random.default_rng(0))
    assert quad.orthant(t, S, st) == pytest.approx(lib, abs=5e-6)


def test_structure_mismatch_is_rejected():
    with pytest.raises(ValueError):
        quad.orthant(np.zeros(3), np.eye(3), {"kind": "equi", "rho": 0.5})


def test_fwer_calibration():
    st = {"kind": "equi", "rho": 0.5}
    S = quad.structured_sigma(3, st)
    w = np.array([0.5, 0.25, 0.25])
    s = quad.calibrate_scale(w, 0.025, S, st)
    assert quad.fwer(quad.thresholds(s, w), S, st) == pytest.approx(0.025, abs=1e-12)
    # correlated tests allow sum(alpha) above the FWER level (Sec. 3 remark)
    assert s > 0.025
    # independent tests: FWER = 1 - prod(1 - alpha_i)
    s0 = quad.calibrate_scale(w, 0.025, np.eye(3), {"kind": "diag"})
    assert 1 - np.prod(1 - s0 * w) == pytest.approx(0.025, abs=1e-12)


def test_information_units_pin():
    with open(os.path.join(GOLDEN, "paper_pins.json")) as f:
        pins = json.load(f)["information_units"]
    for c in pins["cases"]:
        assert round(design.information_units(delta=c["delta"])) == c["I3"]


def test_variance_bound_example_pin():
    with open(os.path.join(GOLDEN, "paper_pins.json")) as f:
        v = json.load(f)["variance_bound_example"]
    assert 1.0 / (4 * v["N1"] * v["N2"]) == pytest.approx(v["bound"], rel=5e-3)


def test_paper_optimal_design_pins():
    # expected power (Eq. 4) with the Gaussian prior of Eq. 10 folded into the
    # sampling law: one orthant probability with covariance Sigma(r) + S Sigma_p S
    with open(os.path.join(GOLDEN, "paper_pins.json")) as f:
        cases = json.load(f)["optimal_designs"]["cases"]
    for c in cases:
        r = np.array(c["r"])
        Delta0 = c["delta0"]["intercept"] + c["delta0"]["slope"] * r
        mu, C = design.collapsed_prior(r, c["I3"], Delta0)
        b = quad.norm_ppf(1.0 - np.array(c["alpha"]))
        p = 1.0 - quad.orthant_dense(b - mu, C)
        assert abs(p - c["power"]) <= c["tol"], (c["name"], p)


def test_smoothness_derivative_d1():
    # Appendix A.3: dP/dalpha = phi(Z_{1-alpha} - m) / phi(Z_{1-alpha}) for one
    # test with a point prior (mean shift m)
    m = 2.1
    for alpha in [0.005, 0.025, 0.1]:
        z = quad.norm_ppf(1 - alpha)
        h = 1e-6

        def P(a):
            return 1 - quad.orthant_dense(np.array([quad.norm_ppf(1 - a) - m]), np.eye(1))
        fd = (P(alpha + h) - P(alpha - h)) / (2 * h)
        assert fd == pytest.approx(quad.norm_pdf(z - m) / quad.norm_pdf(z), rel=1e-6)


def test_analytic_orthant_gradient_matches_fd():
    # d Phi_Sigma(t) / d t_i = phi(t_i) Phi_{Sigma_{-i|i}}(t_{-i} - Sigma_{-i,i} t_i)
    rng = np.random.default_rng(6)
    R = rand_corr(3, rng)
    t = np.array([0.4, 1.1, -0.2])
    h = 1e-5
    for i in range(3):
        e = np.zeros(3)
        e[i] = h
        fd = (quad.orthant_dense(t + e, R) - quad.orthant_dense(t - e, R)) / (2 * h)
        o = [k for k in range(3) if k != i]
        cond = R[np.ix_(o, o)] - np.outer(R[o, i], R[i, o])
        an = quad.norm_pdf(t[i]) * quad.orthant_dense(t[o] - R[o, i] * t[i], cond)
        assert fd == pytest.approx(an, abs=1e-8)
