"""On-device FWER calibration (Eq. 2): each design's alpha split is scaled
until the Monte Carlo FWER under mu = 0 reaches alpha0.  Checked against the
oracle's quadrature calibration (the stored tables), the oracle's
same-stream Monte Carlo at the returned thresholds, and the exact FWER there."""
import numpy as np
import pytest

import workloads
from oracle import quad

from gpu_util import assert_discordance, oracle_same_stream

pytestmark = pytest.mark.gpu
ALPHA0 = workloads.ALPHA0


@pytest.fixture(scope="module")
def ctx():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2005_10494_gb300 as pkg
    return pkg.Context(0)


def calibrate(ctx, prob, w, rounds=14, seed=3):
    import torch

    import paper_2005_10494_gb300 as pkg
    dp = pkg.DeviceProblem.from_workload(prob)
    wt = torch.as_tensor(w, dtype=torch.float64, device="cuda")
    out = pkg.mc_fwer_calibrate(ctx, dp, wt, ALPHA0, rounds=rounds, seed=seed)
    ctx.sync_status()
    return {k: v.cpu().numpy() for k, v in out.items()}


def slope(w, s, Sigma, structure):
    # dFWER/ds at s from the oracle's exact FWER (central difference)
    h = 1e-6 * s
    return (quad.fwer(quad.thresholds(s + h, w), Sigma, structure)
            - quad.fwer(quad.thresholds(s - h, w), Sigma, structure)) / (2 * h)


@pytest.mark.parametrize("config,every,n", [("c2", 4, 4_000_000), ("c4", 16, 2_000_000), ("c5", 32, 1_000_000)])
def test_calibrated_scale_matches_oracle(ctx, config, every, n):
    prob, w, ref, _ = workloads.fwer_calibration(config, n_draws=n, every=every)
    out = calibrate(ctx, prob, w)
    se_f = np.sqrt(ALPHA0 * (1 - ALPHA0) / n)
    d = prob.d_of(0)
    check = range(prob.n_design) if config == "c2" else range(0, prob.n_design, 3)
    for j in check:
        sc = prob.design_scen[j]
        wj = w[j * d:(j + 1) * d]
        g = slope(wj, ref[j], prob.sigmas[sc], prob.structures[sc])
        assert abs(out["scale"][j] - ref[j]) <= 5 * se_f / g + 1e-9, (j, out["scale"][j], ref[j], se_f / g)
        # the last round's estimate sits on the crossing of the step function
        assert abs(out["fwer"][j] - ALPHA0) <= 1e-5, (j, out["fwer"][j])
        # and it is an honest estimate of the exact FWER at the returned scale
        exact = quad.fwer(quad.thresholds(out["scale"][j], wj), prob.sigmas[sc], prob.structures[sc])
        assert abs(out["fwer"][j] - exact) <= 5 * se_f + 1e-7, (j, out["fwer"][j], exact)
    # thresholds are Z_{1 - scale w}
    bt = quad.norm_ppf(1.0 - np.repeat(out["scale"], d) * w)
    np.testing.assert_allclose(out["b"], bt, rtol=1e-12, atol=1e-12)


def test_last_round_is_the_same_stream_estimate(ctx):
    # the returned FWER is hits / N of the returned thresholds on the designs'
    # own stream: the oracle's FP64 Monte Carlo on that stream agrees up to
    # the draws within 1e-4 of a threshold
    prob, w, _, _ = workloads.fwer_calibration("c2", n_draws=200_000, every=8)
    out = calibrate(ctx, prob, w, rounds=10, seed=11)
    d = 3
    cal = workloads.Problem("cal", prob.sigmas, prob.design_scen, [np.zeros(d)] * prob.n_design,
                            [out["b"][j * d:(j + 1) * d] for j in range(prob.n_design)], prob.n_draws, prob.keys)
    idx = list(range(0, prob.n_design, 5))
    hits = np.rint(out["fwer"] * prob.n_draws.astype(np.float64)).astype(np.int64)
    assert_discordance(hits, oracle_same_stream(cal, 11, idx), idx)


def test_single_test_split_is_exact(ctx):
    # one nonzero weight: the bracket is a point, s = alpha0 / w, b = Z_{1 - alpha0}
    prob = workloads.Problem("one", [np.array([[1.0, 0.3], [0.3, 1.0]])], [0, 0], [np.zeros(2)] * 2,
                             [np.zeros(2)] * 2, [100_000, 100_000], [0, 1])
    w = np.array([0.0, 0.5, 2.0, 0.0])
    out = calibrate(ctx, prob, w, rounds=4)
    np.testing.assert_allclose(out["scale"], [ALPHA0 / 0.5, ALPHA0 / 2.0], rtol=1e-15)
    assert np.isinf(out["b"][0]) and np.isinf(out["b"][3])
    np.testing.assert_allclose(out["b"][[1, 2]], quad.norm_ppf(1 - ALPHA0), rtol=1e-13)


def test_invalid_splits_and_arguments(ctx):
    import torch

    import paper_2005_10494_gb300 as pkg
    from paper_2005_10494_gb300.binding import MCD_EINVAL
    prob = workloads.Problem("bad", [np.eye(2)], [0, 0, 0], [np.zeros(2)] * 3, [np.zeros(2)] * 3,
                             [1000] * 3, [0, 1, 2])
    dp = pkg.DeviceProblem.from_workload(prob)
    w = torch.as_tensor([0.5, 0.5, -0.1, 1.0, 0.3, 0.7], dtype=torch.float64, device="cuda")
    out = pkg.mc_fwer_calibrate(ctx, dp, w, ALPHA0, rounds=4)
    with pytest.raises(pkg.MCDError) as e:
        ctx.sync_status()
    assert e.value.code == MCD_EINVAL and e.value.index == 1
    sc = out["scale"].cpu().numpy()
    assert np.isnan(sc[1]) and np.all(np.isfinite(sc[[0, 2]]))
    for kw in ({"rounds": 1}, {"alpha0": 0.0}, {"alpha0": 1.0}):
        args = {"rounds": 4, "alpha0": ALPHA0}
        args.update(kw)
        with pytest.raises(pkg.MCDError) as e:
            pkg.mc_fwer_calibrate(ctx, dp, w, args["alpha0"], rounds=args["rounds"])
        assert e.value.code == MCD_EINVAL
