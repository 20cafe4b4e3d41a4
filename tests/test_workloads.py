"""The seeded input module: design model against the oracle's restatement,
its Jacobian against finite differences, and the stored FWER thresholds
against the oracle's own calibration (Eq. 2)."""
import numpy as np
import pytest

import workloads
from oracle import design, quad


def test_mean_shift_matches_oracle_restatement():
    for d in [3, 10, 20]:
        for q in [0.05, 0.3, 0.95]:
            for dp, dm in [(0.5, 0.1), (0.3, 0.2), (0.8, 0.2)]:
                mu, _, _ = workloads.design_region(q, 0.5, dp, dm, d, 0.03, 0.0)
                np.testing.assert_allclose(mu, design.mean_shift(q, dp, dm, d, 211.0), rtol=1e-15, atol=0)


def test_jacobian_matches_finite_differences():
    tab = workloads.tables()["c4"]
    curve = workloads.ScaleCurve(tab["a"], tab["scale"])
    theta = np.array([0.37, 0.55, 0.5, 0.1])

    def t_of(th):
        s, ds = curve(th[1])
        mu, b, _ = workloads.design_region(th[0], th[1], th[2], th[3], 10, float(s), float(ds))
        return b - mu
    s, ds = curve(theta[1])
    _, _, jac = workloads.design_region(*theta, 10, float(s), float(ds))
    h = 1e-6
    for k in range(4):
        e = np.zeros(4)
        e[k] = h
        fd = (t_of(theta + e) - t_of(theta - e)) / (2 * h)
        np.testing.assert_allclose(jac[:, k], fd, rtol=1e-6, atol=1e-8)


@pytest.mark.parametrize("config", ["c2", "c4", "c5"])
def test_stored_thresholds_satisfy_fwer(config):
    rng = np.random.default_rng(7)
    if config == "c2":
        tab = workloads.tables()["c2"]["scenarios"][3]
        d, st = 3, {"kind": "equi", "rho": tab["rho"]}
    elif config == "c4":
        tab = workloads.tables()["c4"]
        d, st = 10, {"kind": "ar1", "rho": 0.3}
    else:
        tab = workloads.tables()["c5"]
        d, st = 20, {"kind": "block", "sizes": [5, 5, 5, 5], "rho_in": 0.6, "rho_out": 0.1}
    curve = workloads.ScaleCurve(tab["a"], tab["scale"])
    S = quad.structured_sigma(d, st)
    for a in rng.uniform(0.2, 0.8, 2):
        s, _ = curve(a)
        b = quad.thresholds(float(s), workloads.alloc_weights(a, d))
        assert quad.fwer(b, S, st) == pytest.approx(0.025, abs=1e-10)


def test_stored_scale_equals_fresh_oracle_calibration():
    tab = workloads.tables()
    st = {"kind": "equi", "rho": 0.5}
    s = quad.calibrate_scale(np.ones(3) / 3, 0.025, quad.structured_sigma(3, st), st)
    assert tab["c1"]["scale"] == pytest.approx(s, abs=1e-14)
    sc = workloads.c2_scenarios(16)
    for k in [0, 15]:
        assert tab["c2"]["scenarios"][k]["rho"] == sc[k][2]
        a = tab["c2"]["scenarios"][k]["a"][40]
        st = {"kind": "equi", "rho": sc[k][2]}
        s = quad.calibrate_scale(workloads.alloc_weights(a, 3), 0.025, quad.structured_sigma(3, st), st)
        assert tab["c2"]["scenarios"][k]["scale"][40] == pytest.approx(s, abs=1e-14)


def test_config_shapes():
    p1 = workloads.c1()
    assert p1.n_design == 101 and p1.grid == (1, 101) and int(p1.n_draws[0]) == 100_000
    assert len(set(p1.keys.tolist())) == 1
    p2 = workloads.c2(n_scen=2, g1=4, g2=5, n_draws=1000)
    assert p2.n_design == 40 and p2.grid == (4, 5)
    assert p2.params[7][:2] == (pytest.approx(np.linspace(0.05, 0.95, 4)[1]), pytest.approx(np.linspace(0.2, 0.8, 5)[2]))
    p4 = workloads.c4(g1=2, g2=3, n_draws=10)
    assert p4.n_design == 6 and p4.scen_d[0] == 10
    p3 = workloads.c3(n_scen=8)
    assert set(p3.scen_d.tolist()) <= set(range(3, 11))
    assert all(1e5 <= n <= 1e7 for n in p3.n_draws)
    for S in p3.sigmas:
        assert np.allclose(np.diag(S), 1.0) and np.linalg.eigvalsh(S).min() > 0
    assert list(workloads.c5_subsample()) == sorted(set(workloads.c5_subsample()))


def test_c1_surface_has_interior_optimum():
    # the exact success probability over the C1 cutoff grid peaks inside (0.05, 0.95)
    p1 = workloads.c1()
    vals = [1.0 - quad.orthant_equi(p1.t(j), 0.5) for j in range(p1.n_design)]
    k = int(np.argmax(vals))
    assert 0 < k < 100
    assert min(vals) > 0.4 and max(vals) < 0.99


def test_paper_designs_match_oracle_collapse():
    # the input module's sampling law of the paper's designs (Eq. 1, 3, 10)
    # equals the oracle's independent restatement
    p = workloads.paper_optima(n_draws=10)
    r_list = [[1.0], [1.0, 0.365], [1.0, 0.446, 0.168]]
    I3s = [127.0, 211.0, 211.0]
    d0s = [lambda r: 0.25 + 0.0 * r, lambda r: 0.3 - 0.1 * r, lambda r: 0.8 - 0.6 * r]
    for j in range(3):
        r = np.array(r_list[j])
        mu, C = design.collapsed_prior(r, I3s[j], d0s[j](r))
        np.testing.assert_allclose(p.mus[j], mu, rtol=1e-14, atol=0)
        np.testing.assert_allclose(p.sigmas[j], C, rtol=1e-14, atol=1e-15)


def test_split_from_box_maps_the_box_onto_the_simplex():
    """w_1 = u_1, w_j = u_j prod_{l<j} (1 - u_l), w_n = prod (1 - u_l): every
    box point gives a split on the simplex, the corners give its vertices,
    and the map is inverted by u_j = w_j / (1 - w_1 - ... - w_{j-1})."""
    rng = np.random.default_rng(0)
    for n in (2, 3, 5):
        u = rng.uniform(0.0, 1.0, (500, n - 1))
        w = workloads.split_from_box(u)
        assert w.shape == (500, n)
        assert np.all(w >= 0.0)
        np.testing.assert_allclose(w.sum(1), 1.0, rtol=0, atol=1e-14)
        rest = 1.0 - np.concatenate([np.zeros((500, 1)), np.cumsum(w[:, :-1], 1)], 1)
        np.testing.assert_allclose(w[:, :-1] / rest[:, :-1], u, rtol=1e-12, atol=1e-12)
    np.testing.assert_array_equal(workloads.split_from_box([[1.0, 0.3]]), [[1.0, 0.0, 0.0]])
    np.testing.assert_array_equal(workloads.split_from_box([[0.0, 1.0]]), [[0.0, 1.0, 0.0]])
    np.testing.assert_array_equal(workloads.split_from_box([[0.0, 0.0]]), [[0.0, 0.0, 1.0]])


def test_paper_r_pairs_are_the_171_nested_pairs():
    pairs = workloads.paper_r_pairs()
    assert len(pairs) == 171 == 19 * 18 // 2
    assert len(set(pairs)) == 171
    for r2, r3 in pairs:
        assert 0.0 < r3 < r2 < 1.0
        for v in (r2, r3):
            assert abs(v / 0.05 - round(v / 0.05)) < 1e-9
    assert min(b for _, b in pairs) == 0.05 and max(a for a, _ in pairs) == 0.95


def test_box_points_are_seeded_and_uniform():
    a = workloads.box_points(20000, 2, seed=3)
    np.testing.assert_array_equal(a, workloads.box_points(20000, 2, seed=3))
    assert not np.array_equal(a, workloads.box_points(20000, 2, seed=4))
    assert np.all((a >= 0.0) & (a <= 1.0))
    np.testing.assert_allclose(a.mean(0), 0.5, atol=0.01)
    np.testing.assert_allclose(a.var(0), 1.0 / 12.0, atol=0.003)


def test_nested_correlation_matches_patient_level_simulation():
    """Eq. 1 from its construction: the Z statistic of population k is the
    scaled sum of its patients' scores, populations are nested (the first
    n r_k patients), so corr(Z_k, Z_l) = n_l / sqrt(n_k n_l) = sqrt(r_l / r_k).
    Simulated at patient level; the workload's Sigma(r) and the oracle's
    restatement (its collapsed law with a vanishing prior) both match."""
    from oracle import design
    r = np.array([1.0, 0.6, 0.25])
    n = 400
    sizes = (n * r).astype(int)
    rng = np.random.default_rng(11)
    eps = rng.standard_normal((40000, n))
    cs = np.cumsum(eps, axis=1)
    z = np.stack([cs[:, m - 1] / np.sqrt(m) for m in sizes], axis=1)
    emp = np.corrcoef(z, rowvar=False)
    np.testing.assert_allclose(workloads.nested_sigma(r), emp, atol=0.015)
    _, cov = design.collapsed_prior(r, 211.0, [0.2, 0.2, 0.2], prior_sd_scale=1e14)
    np.testing.assert_allclose(cov, workloads.nested_sigma(r), rtol=0, atol=1e-9)
    np.testing.assert_allclose(np.diag(emp), 1.0)


def test_collapsed_prior_covariance_closed_form():
    """With the prior of Eq. 10, sd_i = 1 / sqrt(20 r_i) and prior
    correlation Sigma(r), S_i sd_i = sqrt(I3 / 20) for every population, so
    the folded covariance is Sigma(r) (1 + I3 / 20) and the mean S theta."""
    from oracle import design
    r = np.array([1.0, 0.446, 0.168])
    d0 = np.array([0.2, 0.3, 0.5])
    for I3 in (127.0, 211.0):
        mean, cov = design.collapsed_prior(r, I3, d0)
        np.testing.assert_allclose(cov, workloads.nested_sigma(r) * (1.0 + I3 / 20.0), rtol=1e-13)
        np.testing.assert_allclose(mean, np.sqrt(r * I3) * -np.log1p(-d0), rtol=1e-14)


@pytest.mark.parametrize("d,eta", [(3, 1.0), (4, 2.0), (6, 2.0)])
def test_lkj_cvine_off_diagonal_marginal(d, eta):
    """Lewandowski, Kurowicka and Joe (2009): under LKJ(eta) in dimension d
    every off-diagonal correlation is marginally Beta(b, b) on (-1, 1) with
    b = eta - 1 + d / 2, whose variance is 1 / (2 b + 1)."""
    from scipy import stats
    rng = np.random.default_rng(17)
    b = eta - 1.0 + d / 2.0
    mats = [workloads.lkj_cvine(d, eta, rng) for _ in range(3000)]
    for M in mats[:50]:
        np.testing.assert_allclose(M, M.T)
        np.testing.assert_allclose(np.diag(M), 1.0)
        assert np.linalg.eigvalsh(M).min() > 0
    iu = np.triu_indices(d, 1)
    for i, j in zip(*iu):
        x = np.array([M[i, j] for M in mats])
        res = stats.kstest((x + 1.0) / 2.0, stats.beta(b, b).cdf)
        assert res.pvalue > 1e-3, (d, eta, i, j, res)
        assert abs(x.var() - 1.0 / (2 * b + 1)) < 0.1 / (2 * b + 1)
