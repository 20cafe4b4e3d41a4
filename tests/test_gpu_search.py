"""The d=10 configuration's design search: gradient ascent driven by the
adjoint against grid + local-quadratic smoothing + argmax, both evaluated by the
exact objective (AR(1) Markov-recursion quadrature)."""
import numpy as np
import pytest

import workloads
from oracle import quad

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2005_10494_gb300 as pkg
    return pkg.Context(0)


def exact(q, a):
    mu, b, _ = workloads.design_at("c4", q, a)
    return 1.0 - quad.orthant_ar1(b - mu, 0.3)


def test_c4_gradient_search_vs_grid_smoothing(ctx):
    from paper_2005_10494_gb300 import search
    prob = workloads.c4(keys="crn")                        # 32 x 32 grid, 1e7 draws per design
    qs, as_ = np.linspace(0.05, 0.95, 32), np.linspace(0.2, 0.8, 32)
    gi, gj, _ = search.grid_argmax(ctx, prob, 32, 32)
    grid_exact = np.array([exact(q, a) for q in qs for a in as_]).reshape(32, 32)
    best = grid_exact.max()

    x, p_hat, hist = search.gradient_search(ctx, lambda x: workloads.design_at("c4", x[0], x[1]),
                                            prob.sigmas[0], x0=(0.5, 0.5), lo=(0.05, 0.2), hi=(0.95, 0.8),
                                            n_draws=10_000_000, steps=120)
    p_search = exact(*x)
    p_grid = grid_exact[gi, gj]
    # SE of one estimate at p ~ 0.9995 and 1e7 draws is about 7e-6
    assert p_search >= best - 3e-5, (x, p_search, best)
    assert p_grid >= best - 3e-5, ((qs[gi], as_[gj]), p_grid, best)
    # the search moved uphill from its start
    assert p_search > exact(0.5, 0.5)
    assert abs(p_hat - p_search) <= 5 * np.sqrt(p_search * (1 - p_search) / 1e7) + 1e-7


def _c1_region(x):
    t = workloads.tables()["c1"]
    mu, b, jac = workloads.design_region(float(x[0]), 2.0 / 3.0, 0.5, 0.1, 3, t["scale"], 0.0)
    return mu, b, jac


def _c1_exact(q):
    mu, b, _ = _c1_region([q])
    return 1.0 - quad.orthant_equi(b - mu, 0.5)


def test_c1_gradient_search_finds_the_interior_optimum(ctx):
    """The d=3 cutoff curve (equicorrelation 0.5, common critical value) has
    an interior maximum near q = 0.69.  Started 38 grid steps away, the
    adjoint-driven search must end within one grid step (0.009) of the exact
    maximiser of the quadrature objective, with exact power within 2 SE of
    the best."""
    from scipy.optimize import minimize_scalar

    from paper_2005_10494_gb300 import search
    best = minimize_scalar(lambda q: -_c1_exact(q), bounds=(0.05, 0.95), method="bounded",
                           options={"xatol": 1e-9})
    q_star, p_star = float(best.x), -float(best.fun)
    assert 0.6 < q_star < 0.8
    x0 = 0.35
    assert abs(x0 - q_star) > 10 * 0.009
    n = 10_000_000
    x, p_hat, hist = search.gradient_search(ctx, _c1_region, workloads.equicorrelated(3, 0.5), x0=(x0,),
                                            lo=(0.05,), hi=(0.95,), n_draws=n, steps=120)
    se = np.sqrt(p_star * (1 - p_star) / n)
    assert abs(x[0] - q_star) <= 0.009, (x, q_star)
    assert _c1_exact(x[0]) >= p_star - 2 * se, (x, _c1_exact(x[0]), p_star)


def test_c2_gradient_search_interior_cutoff(ctx):
    """A d=3 grid scenario (delta+ 0.31, delta- 0.16, rho 0.66) whose exact
    optimum lies on the allocation edge a = 0.8 with an interior cutoff
    quantile: the projected search, started 20 grid steps away in q and
    inside in a, must reach the edge and a cutoff within one grid step
    (0.9 / 63) of the exact maximiser."""
    from scipy.optimize import minimize_scalar

    from paper_2005_10494_gb300 import search
    s = 1
    rho = workloads.c2_scenarios(16)[s][2]

    def region(x):
        return workloads.design_at("c2", float(x[0]), float(x[1]), scenario=s)

    def exact(q, a):
        mu, b, _ = region((q, a))
        return 1.0 - quad.orthant_equi(b - mu, rho)

    best = minimize_scalar(lambda q: -exact(q, 0.8), bounds=(0.05, 0.95), method="bounded",
                           options={"xatol": 1e-9})
    q_star, p_star = float(best.x), -float(best.fun)
    assert 0.2 < q_star < 0.6
    assert exact(q_star, 0.8) > exact(q_star, 0.79)         # the allocation edge binds
    step = 0.9 / 63
    x0 = (min(0.95, q_star + 20 * step), 0.5)
    n = 10_000_000
    x, p_hat, hist = search.gradient_search(ctx, region, workloads.equicorrelated(3, rho), x0=x0,
                                            lo=(0.05, 0.2), hi=(0.95, 0.8), n_draws=n, steps=150)
    se = np.sqrt(p_star * (1 - p_star) / n)
    assert abs(x[0] - q_star) <= step, (x, q_star)
    assert x[1] >= 0.8 - 1e-3, x
    assert exact(*x) >= p_star - 2 * se, (x, exact(*x), p_star)
