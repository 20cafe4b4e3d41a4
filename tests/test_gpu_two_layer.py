"""The paper's two-layer estimator (Sec. 2.2, Eq. 5-7) on the GPU: N1 outer
prior samples share one inner stream of N2 draws (the shared-draw kernel,
one design per outer sample).  Checks: hits bit-identical to the per-design
kernel and within the oracle's same-stream band; over seeds, the mean of the
estimate matches the exact expected power and its variance the exact
variance of the cross-paired estimator (not Appendix A.2's 1/(4 N1 N2))."""
import numpy as np
import pytest

import workloads
from oracle import design

from gpu_util import assert_discordance, oracle_same_stream, run

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2005_10494_gb300 as pkg
    return pkg.Context(0)


def test_two_layer_hits_identical_and_same_stream(ctx):
    prob = workloads.paper_two_layer("c", N1=2048, N2=20480, seed=3, key=9)
    sh = run(ctx, prob, seed=4, shared=True)
    per = run(ctx, prob, seed=4)
    np.testing.assert_array_equal(sh["hits"], per["hits"])
    idx = sorted(np.random.default_rng(1).choice(prob.n_design, 16, replace=False).tolist())
    assert_discordance(sh["hits"], oracle_same_stream(prob, 4, idx), idx)


@pytest.mark.parametrize("cond,N1,N2,reps", [("c", 512, 2048, 160), ("a", 256, 1024, 160)])
def test_two_layer_mean_and_variance_over_seeds(ctx, cond, N1, N2, reps):
    import torch

    import paper_2005_10494_gb300 as pkg
    r, alpha, I3, d0 = workloads.PAPER_CONDITIONS[cond]
    m = design.two_layer_moments(r, alpha, I3, d0)
    V = design.two_layer_variance(N1, N2, m)
    prob = workloads.paper_two_layer(cond, N1=N1, N2=N2, seed=0, key=0)
    dp = pkg.DeviceProblem.from_workload(prob)
    plan = pkg.Plan(ctx, dp, shared=True)
    est = []
    for rep in range(reps):
        a = workloads.paper_two_layer_arrays(cond, N1=N1, N2=N2, seed=1000 + rep, key=0)
        dp.mu.copy_(torch.as_tensor(a["mu"].ravel(), dtype=torch.float64))     # new outer samples
        out = plan.eval(seed=rep)                                               # new inner draws
        est.append(float(out["p"].mean().item()))
    ctx.sync_status()
    plan.close()
    est = np.array(est)
    assert abs(est.mean() - m[0]) <= 5 * np.sqrt(V / reps)
    # sample variance of `reps` estimates: relative SE about sqrt(2 / reps)
    # (about 0.11) for near-normal estimates; 4 of those either side
    ratio = est.var(ddof=1) / V
    assert 0.55 <= ratio <= 1.6, (ratio, est.var(ddof=1), V)
    assert V > 10 * (1.0 / (4 * N1 * N2))


def test_two_layer_paper_size(ctx):
    # N1 = 10240 outer x N2 = 20480 inner samples (Sec. 2.2): one estimate of
    # the strong-biomarker optimum, within 5 SD of the exact expected power
    r, alpha, I3, d0 = workloads.PAPER_CONDITIONS["c"]
    m = design.two_layer_moments(r, alpha, I3, d0)
    prob = workloads.paper_two_layer("c", N1=10240, N2=20480, seed=5, key=2)
    out = run(ctx, prob, seed=6, shared=True)
    P_hat = float(out["p"].mean())
    assert abs(P_hat - m[0]) <= 5 * np.sqrt(design.two_layer_variance(10240, 20480, m))
