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
