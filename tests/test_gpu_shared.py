"""The shared-draw path (designs with common random numbers evaluated
against one generated stream): hit counts bit-identical to the per-design
kernel and to the oracle's same-stream band, gradients equal up to FP32
summation order, error paths."""
import numpy as np
import pytest

import workloads

from gpu_util import assert_discordance, oracle_same_stream, run

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2005_10494_gb300 as pkg
    return pkg.Context(0)


def _grad_close(a, b):
    # same draws, same estimator; the FP32 sums differ only in addition order.
    # grad_se is a batch-means estimate over each path's own tiles (NaN with a
    # single batch; under common random numbers its error is shared by all
    # designs of a group), so it only scales the tolerance here; its
    # calibration has a test of its own
    sa, sb = a["grad_se"], b["grad_se"]
    se = np.fmax(np.nan_to_num(sa, nan=0.0), np.nan_to_num(sb, nan=0.0))
    for name in ["grad_lr", "grad_sig"]:
        if name in b:
            tol = 0.02 * se + 1e-6 * np.maximum(1.0, np.abs(b[name])) + 1e-7
            bad = np.flatnonzero(~(np.abs(a[name] - b[name]) <= tol))
            assert bad.size == 0, (name, bad[:5], a[name][bad[:5]], b[name][bad[:5]])


@pytest.mark.parametrize("d_list", [(1, 2, 3, 4), (5, 7, 8, 10), (13, 16, 20)])
def test_shared_hits_identical_to_per_design(ctx, d_list):
    prob = workloads.crn_groups(np.random.default_rng(sum(d_list)), d_list=d_list, group=40, extra=3,
                                n_draws=20_011, draw_begin=7)
    per = run(ctx, prob, seed=5)
    sh = run(ctx, prob, seed=5, shared=True)
    np.testing.assert_array_equal(sh["hits"], per["hits"])
    np.testing.assert_array_equal(sh["p"], per["p"])
    np.testing.assert_array_equal(sh["se"], per["se"])


def test_shared_several_chunks_and_tail(ctx):
    # 2600 designs of d = 3 (three chunks), draw count not a multiple of a batch
    prob = workloads.crn_groups(np.random.default_rng(11), d_list=(3,), group=2600, extra=0,
                                n_draws=70_001, draw_begin=1)
    per = run(ctx, prob, seed=2)
    sh = run(ctx, prob, seed=2, shared=True, graph=True)
    np.testing.assert_array_equal(sh["hits"], per["hits"])
    idx = sorted(np.random.default_rng(0).choice(prob.n_design, 12, replace=False).tolist())
    assert_discordance(sh["hits"], oracle_same_stream(prob, 2, idx), idx)


@pytest.mark.parametrize("d_list", [(3,), (10,), (20,)])
def test_shared_gradients_match_per_design(ctx, d_list):
    prob = workloads.crn_groups(np.random.default_rng(3 + d_list[0]), d_list=d_list, group=70, extra=2,
                                n_draws=100_003, draw_begin=5)
    per = run(ctx, prob, seed=1, grad=True, h=0.05)
    sh = run(ctx, prob, seed=1, grad=True, h=0.05, shared=True)
    np.testing.assert_array_equal(sh["hits"], per["hits"])
    _grad_close(sh, per)
    per0 = run(ctx, prob, seed=1, grad=True)
    sh0 = run(ctx, prob, seed=1, grad=True, shared=True)
    np.testing.assert_array_equal(sh0["hits"], per0["hits"])
    _grad_close(sh0, per0)


def test_shared_gradients_against_oracle_same_stream(ctx):
    from oracle import mc as omc
    prob = workloads.crn_groups(np.random.default_rng(21), d_list=(3,), group=48, extra=0, n_draws=30_000,
                                draw_begin=0)
    h = 0.05
    sh = run(ctx, prob, seed=4, grad=True, h=h, shared=True)
    idx = [0, 17, 47]
    ora = oracle_same_stream(prob, 4, idx, grad=True, h=h)
    assert_discordance(sh["hits"], ora, idx)
    S = prob.sigmas[0]
    Linv = np.linalg.inv(omc.cholesky(S))
    n = 30_000
    for k, j in enumerate(idx):
        g_ref = omc.lr_gradient_mu(S, ora["A"][k], ora["B"][k], ora["hits"][k], n)
        amb = int(ora["ambiguous"][k])
        # the bound of the per-design same-stream test: flipped draws and FP32 normals
        bound = np.abs(Linv.T).sum(axis=1) * (12.0 * amb + 4.0 * n * 2e-5 + amb * np.abs(ora["B"][k]).max() / n) / n
        np.testing.assert_array_less(np.abs(sh["grad_lr"][3 * j:3 * j + 3] - g_ref), bound + 1e-9)
        np.testing.assert_allclose(sh["grad_sig"][3 * j:3 * j + 3], ora["G"][k] / n, rtol=2e-3, atol=2e-4)


def test_shared_c2_full_identical_to_per_design(ctx):
    # the benchmark configuration: 16 scenarios x 4096 designs x 1e6 draws,
    # gradients with the sigmoid bandwidth 1e-2
    prob = workloads.c2()
    jac = prob.jac_packed()
    per = run(ctx, prob, seed=0, grad=True, k=4, jac=jac, h=0.01, graph=True)
    sh = run(ctx, prob, seed=0, grad=True, k=4, jac=jac, h=0.01, graph=True, shared=True)
    np.testing.assert_array_equal(sh["hits"], per["hits"])
    _grad_close(sh, per)


def test_shared_error_paths(ctx):
    import paper_2005_10494_gb300 as pkg
    from paper_2005_10494_gb300.binding import MCD_ENAN, MCD_ENOTSPD, MCD_EUNSUPPORTED
    bad = np.array([[1.0, 2.0], [2.0, 1.0]])
    n = 40
    prob = workloads.Problem("bad", [np.eye(2), bad], [0] * n + [1] * n, [np.zeros(2)] * (2 * n),
                             [np.ones(2)] * (2 * n), [1000] * (2 * n), [0] * n + [1] * n)
    dp = pkg.DeviceProblem.from_workload(prob)
    plan = pkg.Plan(ctx, dp, shared=True)
    out = plan.eval(0)
    with pytest.raises(pkg.MCDError) as e:
        ctx.sync_status()
    assert e.value.code == MCD_ENOTSPD and e.value.index == 1
    hits = out["hits"].cpu().numpy()
    assert np.all(hits[n:] == 0) and np.all(hits[:n] > 0)
    plan.close()
    mus = [np.zeros(2) for _ in range(n)]
    mus[13] = np.array([0.0, np.nan])
    prob = workloads.Problem("nan", [np.eye(2)], [0] * n, mus, [np.ones(2)] * n, [100] * n, [0] * n)
    dp = pkg.DeviceProblem.from_workload(prob)
    pkg.Plan(ctx, dp, shared=True).eval(0)
    with pytest.raises(pkg.MCDError) as e:
        ctx.sync_status()
    assert e.value.code == MCD_ENAN and e.value.index == 13
    with pytest.raises(pkg.MCDError) as e:
        pkg.Plan(ctx, dp, shared=True, fp64=True)
    assert e.value.code == MCD_EUNSUPPORTED


@pytest.mark.parametrize("shared", [False, True])
def test_gradient_se_is_calibrated_across_seeds(ctx, shared):
    # the batch-means standard error against the spread of the estimate over
    # independent seeds, pooled over designs and parameters
    import torch

    import paper_2005_10494_gb300 as pkg
    prob = workloads.c2(n_scen=1, g1=8, g2=8, n_draws=400_000)
    dp = pkg.DeviceProblem.from_workload(prob)
    plan = pkg.Plan(ctx, dp, grad=True, k=4, shared=shared)
    jac = torch.as_tensor(prob.jac_packed(), dtype=torch.float64, device="cuda")
    gs, ses = [], []
    for seed in range(40):
        out = plan.grad(seed, jac, 0.0)
        gs.append(out["grad_lr"].cpu().numpy().copy())
        ses.append(out["grad_se"].cpu().numpy().copy())
    ctx.sync_status()
    plan.close()
    emp = np.array(gs).std(axis=0, ddof=1)
    rep = np.sqrt(np.mean(np.array(ses) ** 2, axis=0))
    ok = emp > 0
    ratio = float(np.median(rep[ok] / emp[ok]))
    assert 0.85 < ratio < 1.15, ratio


@pytest.mark.parametrize("d_list", [(1, 2, 3, 4), (5, 6, 7, 8), (9, 11, 12, 13), (14, 15, 16, 17), (18, 19, 20)])
def test_shared_adjoint_hits_identical_to_per_design(ctx, d_list):
    """The adjoint form of the shared-draw kernel counts its hits in the
    padded slot of the sum A when d is not a multiple of 4 (and by integer
    adds otherwise): the counts equal the per-design kernel's at every d."""
    prob = workloads.crn_groups(np.random.default_rng(50 + sum(d_list)), d_list=d_list, group=36, extra=2,
                                n_draws=30_011, draw_begin=3)
    per = run(ctx, prob, seed=8, grad=True, h=0.02)
    sh = run(ctx, prob, seed=8, grad=True, h=0.02, shared=True)
    np.testing.assert_array_equal(sh["hits"], per["hits"])
    np.testing.assert_array_equal(sh["p"], per["p"])
    _grad_close(sh, per)
