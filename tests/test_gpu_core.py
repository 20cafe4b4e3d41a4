"""GPU parity of the sampling path against the FP64 oracle (through the C ABI)."""
import math

import numpy as np
import pytest

import workloads
from oracle import mc as omc
from oracle import quad, smooth

from gpu_util import EPS32, EPS64, assert_band, assert_discordance, oracle_same_stream, run

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2005_10494_gb300 as pkg
    return pkg.Context(0)


# ------------------------------------------------------------------ streams
@pytest.mark.parametrize("seed,key,m0", [(0, 0, 0), (1, 7, 3), (2**63 + 5, 2**40 + 3, (2**32 - 3) * 4 + 1),
                                         (0xDEADBEEFCAFEF00D, 0xFFFFFFFFFFFFFFFF, 2**36 - 7)])
def test_philox_words_bit_exact(ctx, seed, key, m0):
    import paper_2005_10494_gb300 as pkg
    count = 4096
    z32, z64, words = pkg.debug_normals(ctx, seed, key, m0, count)
    ctx.sync_status()
    w = words.cpu().numpy().view(np.uint32)
    ref = omc.philox_stream(seed, key, m0 >> 2, len(w) // 4)
    np.testing.assert_array_equal(w, ref)


def test_normals_match_oracle(ctx):
    import paper_2005_10494_gb300 as pkg
    seed, key, count = 123, 456, 1 << 20
    z32, z64, _ = pkg.debug_normals(ctx, seed, key, 0, count)
    ctx.sync_status()
    ref = omc.normals(seed, key, 0, count)
    e64 = np.abs(z64.cpu().numpy() - ref)
    e32 = np.abs(z32.cpu().numpy().astype(np.float64) - ref)
    assert e64.max() < 1e-13
    # FP32 path: radius error below 4e-6 (2v near u0 = 1, hardware log2
    # elsewhere), angle error below ~1.3e-6 rad (FP32 angle and approximate
    # sin / cos) times |r| <= 5.77
    assert e32.max() < 1.2e-5
    assert e32.mean() < 2e-6


# -------------------------------------------------------------- C1 parity
@pytest.mark.parametrize("keys", ["crn", "independent"])
def test_c1_same_stream_and_exact(ctx, keys):
    prob = workloads.c1(keys=keys)
    out = run(ctx, prob, seed=0)
    idx = list(range(prob.n_design))
    ora = oracle_same_stream(prob, 0, idx)
    assert_discordance(out["hits"], ora, idx)
    n = int(prob.n_draws[0])
    exact = [1.0 - quad.orthant_equi(prob.t(j), 0.5) for j in idx]
    assert_band(out["p"], exact, n, idx)
    assert np.all((out["p"] >= 0) & (out["p"] <= 1))
    np.testing.assert_allclose(out["se"], np.sqrt(out["p"] * (1 - out["p"]) / n), rtol=1e-12, atol=0)


def test_c1_argmax_within_one_step(ctx):
    import torch

    import paper_2005_10494_gb300 as pkg
    prob = workloads.c1(keys="crn")
    out = run(ctx, prob, seed=0)
    p = torch.as_tensor(out["p"], dtype=torch.float64, device="cuda")
    r = pkg.mc_smooth_argmax(ctx, p, 1, 1, prob.n_design, bandwidth=3.0, degree=2)
    ctx.sync_status()
    exact = [1.0 - quad.orthant_equi(prob.t(j), 0.5) for j in range(prob.n_design)]
    assert abs(int(r["argmax_idx"].item()) - int(np.argmax(exact))) <= 1


def test_reruns_are_bit_identical(ctx):
    prob = workloads.c2(n_scen=2, g1=5, g2=6, n_draws=30_000)
    a = run(ctx, prob, seed=9, grad=True, k=4, jac=prob.jac_packed(), h=0.01)
    b = run(ctx, prob, seed=9, grad=True, k=4, jac=prob.jac_packed(), h=0.01)
    for name in a:
        np.testing.assert_array_equal(a[name], b[name])
    c = run(ctx, prob, seed=9, graph=True)
    np.testing.assert_array_equal(a["hits"], c["hits"])
    d = run(ctx, prob, seed=10)
    assert not np.array_equal(a["hits"], d["hits"])


def test_graph_replay_with_timing(ctx):
    import torch

    import paper_2005_10494_gb300 as pkg
    prob = workloads.c2(n_scen=1, g1=4, g2=4, n_draws=200_000)
    dp = pkg.DeviceProblem.from_workload(prob)
    jac = torch.as_tensor(prob.jac_packed(), dtype=torch.float64, device="cuda")
    plain = pkg.Plan(ctx, dp, grad=True, k=4)
    ref = {k: v.cpu().numpy() for k, v in plain.grad(5, jac, 0.01).items()}
    plan = pkg.Plan(ctx, dp, grad=True, k=4, graph=True, timing=True)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    for seed in (4, 5, 5):                     # capture, re-capture on a new seed, replay
        out = plan.grad(seed, jac, 0.01, stream=s)
        assert plan.kernel_ms() > 0.0
    s.synchronize()
    ctx.sync_status()
    for k in ref:
        np.testing.assert_array_equal(out[k].cpu().numpy(), ref[k])


def test_one_shot_equals_plan(ctx):
    import paper_2005_10494_gb300 as pkg
    prob = workloads.c1(n_draws=5000, keys="independent")
    dp = pkg.DeviceProblem.from_workload(prob)
    one = pkg.mc_design_eval(ctx, dp, 4)
    ctx.sync_status()
    plan = run(ctx, prob, seed=4)
    np.testing.assert_array_equal(one["hits"].cpu().numpy(), plan["hits"])


def test_injected_launch_failure(ctx):
    """Host-side fault injection (no GPU fault): the next launch returns
    MCD_ECUDA with the injected error's text and queues nothing; the plan,
    the one-shot call and the context stay usable and give the same counts."""
    import torch

    import paper_2005_10494_gb300 as pkg
    from paper_2005_10494_gb300.binding import MCD_ECUDA, MCD_EINVAL
    prob = workloads.c1(n_draws=5000, keys="independent")
    dp = pkg.DeviceProblem.from_workload(prob)
    plan = pkg.Plan(ctx, dp, graph=False)
    ref = plan.eval(4)["hits"].clone()
    ctx.sync_status()
    ctx.fail_next_launch(9)
    with pytest.raises(pkg.MCDError) as e:
        plan.eval(4)
    assert e.value.code == MCD_ECUDA and "injected" in str(e.value)
    assert torch.equal(plan.eval(4)["hits"], ref)
    ctx.sync_status()
    ctx.fail_next_launch(2)
    with pytest.raises(pkg.MCDError) as e:
        pkg.mc_design_eval(ctx, dp, 4)
    assert e.value.code == MCD_ECUDA
    assert torch.equal(pkg.mc_design_eval(ctx, dp, 4)["hits"], ref)
    ctx.sync_status()
    ctx.fail_next_launch(9)
    ctx.fail_next_launch(0)            # cleared before any launch
    assert torch.equal(plan.eval(4)["hits"], ref)
    ctx.sync_status()
    with pytest.raises(pkg.MCDError) as e:
        ctx.fail_next_launch(-1)
    assert e.value.code == MCD_EINVAL
    plan.close()


def test_plan_destroyed_after_its_context(ctx):
    """A plan may outlive its context (a garbage collector can finalise the
    two in either order): destroying it reads nothing of the freed context
    and leaves no CUDA error behind for the next call."""
    import torch

    import paper_2005_10494_gb300 as pkg
    prob = workloads.c1(n_draws=5000, keys="independent")
    dp = pkg.DeviceProblem.from_workload(prob)
    ref = pkg.mc_design_eval(ctx, dp, 6)["hits"].clone()
    ctx.sync_status()
    for _ in range(3):
        c2 = pkg.Context(0)
        plan = pkg.Plan(c2, dp)
        assert torch.equal(plan.eval(6)["hits"], ref)
        c2.sync_status()
        c2.close()                      # the context first ...
        plan.close()                    # ... then its plan
    x = torch.as_tensor(np.random.default_rng(0).random((1, 40, 2)), dtype=torch.float64, device="cuda")
    y = torch.sin(x[..., 0]).contiguous()
    pkg.mc_tps_fit(ctx, x, y, smoothing=1e-6)   # checks for launch errors
    assert torch.equal(pkg.mc_design_eval(ctx, dp, 6)["hits"], ref)
    ctx.sync_status()


# ------------------------------------------------- uneven / ragged problems
@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_random_problems_same_stream(ctx, seed):
    rng = np.random.default_rng(100 + seed)
    prob = workloads.random_problem(rng, n_scen=5, designs_per=(1, 5), n_draws=(0, 40_000))
    out = run(ctx, prob, seed=seed)
    idx = list(range(prob.n_design))
    ora = oracle_same_stream(prob, seed, idx)
    assert_discordance(out["hits"], ora, idx)
    below = run(ctx, prob, seed=seed, region=1)
    np.testing.assert_array_equal(below["hits"], prob.n_draws.astype(np.int64) - out["hits"])
    zero = prob.n_draws == 0
    assert np.all(out["p"][zero] == 0.0)


def test_every_dimension_same_stream(ctx):
    # one design per d = 1..20, uneven draw counts with ragged tails
    rng = np.random.default_rng(7)
    sigmas, mus, bs, scen, nd = [], [], [], [], []
    for d in range(1, 21):
        sigmas.append(workloads.lkj_cvine(d, 2.0, rng) if d > 1 else np.eye(1))
        mus.append(rng.normal(0.4, 0.5, d))
        bs.append(np.full(d, 1.8))
        scen.append(d - 1)
        nd.append(int(rng.integers(20_000, 60_000)))
    prob = workloads.Problem("dims", sigmas, scen, mus, bs, nd, np.arange(20) + 11)
    out = run(ctx, prob, seed=5)
    idx = list(range(20))
    assert_discordance(out["hits"], oracle_same_stream(prob, 5, idx), idx)


def test_draw_range_chunks_add_exactly(ctx):
    prob = workloads.c1(n_draws=200_003, keys="independent").subset([10, 60])
    whole = run(ctx, prob, seed=3)["hits"]
    parts = np.zeros(2, np.int64)
    start = 0
    for n in [1, 65_535, 100_000, 34_467]:
        sub = workloads.c1(n_draws=n, keys="independent").subset([10, 60])
        sub.draw_begin = np.full(2, start, np.uint64)
        parts += run(ctx, sub, seed=3)["hits"]
        start += n
    np.testing.assert_array_equal(parts, whole)


def test_batching_and_tiling_do_not_change_hits(ctx):
    big = workloads.c2(n_scen=3, g1=6, g2=7, n_draws=70_001)
    a = run(ctx, big, seed=1)
    sub_idx = [0, 50, 125]
    b = run(ctx, big.subset(sub_idx), seed=1)
    np.testing.assert_array_equal(a["hits"][sub_idx], b["hits"])
    c = run(ctx, big, seed=1, autotune=True)
    np.testing.assert_array_equal(a["hits"], c["hits"])


def test_large_stream_offsets(ctx):
    # draws near the 2^32 boundary of the Philox call index
    prob = workloads.c1(n_draws=50_000, keys="independent").subset([5, 90])
    prob.draw_begin = np.array([(2**32 // 3) * 4 - 20_000, 2**40 + 12345], np.uint64)
    out = run(ctx, prob, seed=8)
    assert_discordance(out["hits"], oracle_same_stream(prob, 8, [0, 1]), [0, 1])


# ------------------------------------------------------------ FP64 path
@pytest.mark.parametrize("d", [3, 10, 20])
def test_fp64_path_matches_oracle(ctx, d):
    rng = np.random.default_rng(d)
    S = workloads.lkj_cvine(d, 2.0, rng)
    mus = [rng.normal(0.3, 0.3, d) for _ in range(4)]
    bs = [np.full(d, quad.norm_ppf(1 - 0.025 / d)) for _ in range(4)]
    prob = workloads.Problem("fp64", [S], [0] * 4, mus, bs, [30_000] * 4, [1, 2, 3, 4])
    out = run(ctx, prob, seed=2, fp64=True)
    ora = oracle_same_stream(prob, 2, range(4), eps=EPS64)
    assert_discordance(out["hits"], ora, list(range(4)))


# -------------------------------------------------------------- gradients
def test_gradient_sums_same_stream(ctx):
    rng = np.random.default_rng(3)
    prob = workloads.random_problem(rng, n_scen=3, designs_per=(2, 3), d_choices=(2, 3, 5, 8),
                                    n_draws=(50_000, 80_000))
    h = 0.02
    out = run(ctx, prob, seed=6, grad=True, k=0, h=h)
    idx = list(range(prob.n_design))
    ora = oracle_same_stream(prob, 6, idx, grad=True, h=h)
    off = 0
    for k, j in enumerate(idx):
        d = prob.d_of(j)
        n = int(prob.n_draws[j])
        S = prob.sigmas[prob.design_scen[j]]
        g_ref = omc.lr_gradient_mu(S, ora["A"][k], ora["B"][k], ora["hits"][k], n)
        Linv = np.linalg.inv(omc.cholesky(S))
        amb = int(ora["ambiguous"][k])
        # flipped draws move A by |z| <= 5.8 each and p_hat by 1/N; FP32 normals
        # move each sum by at most N * 2e-5
        bound = np.abs(Linv.T).sum(axis=1) * (12.0 * amb + 4.0 * n * 2e-5 + amb * np.abs(ora["B"][k]).max() / n) / n
        np.testing.assert_array_less(np.abs(out["grad_lr"][off:off + d] - g_ref), bound + 1e-9)
        g_sig_ref = ora["G"][k] / n          # the oracle's G already carries the 1/h
        np.testing.assert_allclose(out["grad_sig"][off:off + d], g_sig_ref, rtol=2e-3, atol=2e-4)
        off += d


def test_gradient_vs_finite_differences_c2(ctx):
    prob = workloads.c2(n_scen=2, g1=8, g2=8, n_draws=1_000_000)
    out = run(ctx, prob, seed=11, grad=True, k=4, jac=prob.jac_packed(), h=0.01)
    sc = workloads.c2_scenarios(2)
    rng = np.random.default_rng(0)
    for j in rng.choice(prob.n_design, 6, replace=False):
        s = int(prob.design_scen[j])
        q, a, dp, dm = prob.params[j]
        st = {"kind": "equi", "rho": sc[s][2]}
        from oracle import design
        fd = design.objective_fd_gradient((q, a, dp, dm), 3, 211.0, 0.025,
                                          quad.structured_sigma(3, st), st, step=1e-4)
        g = out["grad_lr"][4 * j:4 * j + 4]
        se = out["grad_se"][4 * j:4 * j + 4]
        tol = np.maximum(np.maximum(0.02 * np.abs(fd), 5 * se), 1e-6)
        assert np.all(np.abs(g - fd) <= tol), (j, g, fd, se)
        gs = out["grad_sig"][4 * j:4 * j + 4]
        tol_s = np.maximum(0.05 * np.abs(fd), 20 * se + 2e-3)
        assert np.all(np.abs(gs - fd) <= tol_s), (j, gs, fd)


def test_autograd_function(ctx):
    import torch

    import paper_2005_10494_gb300 as pkg
    from paper_2005_10494_gb300.autograd import design_eval
    prob = workloads.c1(n_draws=20_000, keys="independent").subset([3, 40, 77])
    dp = pkg.DeviceProblem.from_workload(prob)
    plan = pkg.Plan(ctx, dp, grad=True, k=0)
    mu = dp.mu.requires_grad_(True)
    b = dp.b.requires_grad_(True)
    p = design_eval(mu, b, plan, 0)
    w = torch.tensor([1.0, -2.0, 0.5], dtype=torch.float64, device="cuda")
    (p * w).sum().backward()
    ref = plan.grad(0)["grad_lr"]
    idx = torch.repeat_interleave(torch.arange(3, device="cuda"), 3)
    torch.testing.assert_close(mu.grad, w[idx] * ref)
    torch.testing.assert_close(b.grad, -w[idx] * ref)


# -------------------------------------------------------------- smoothing
@pytest.mark.parametrize("shape,bw,deg", [((1, 101), 3.0, 2), ((64, 64), 3.0, 2), ((37, 150), 3.0, 2),
                                          ((5, 5), 3.0, 2), ((130, 9), 2.5, 1), ((1, 7), 4.0, 0),
                                          ((200, 1), 3.5, 2)])
def test_smoothing_matches_oracle(ctx, shape, bw, deg):
    import torch

    import paper_2005_10494_gb300 as pkg
    g1, g2 = shape
    S = 3
    rng = np.random.default_rng(g1 * 1000 + g2)
    i, j = np.meshgrid(np.arange(g1), np.arange(g2), indexing="ij")
    vals = np.stack([0.7 - 0.0004 * (i - g1 / 3) ** 2 - 0.0002 * (j - g2 / 2) ** 2 + rng.normal(0, 0.01, (g1, g2))
                     for _ in range(S)])
    v = torch.as_tensor(vals.ravel(), dtype=torch.float64, device="cuda")
    r = pkg.mc_smooth_argmax(ctx, v, S, g1, g2, bandwidth=bw, degree=deg, raw=True)
    ctx.sync_status()
    r2 = pkg.mc_smooth_argmax(ctx, v, S, g1, g2, bandwidth=bw, degree=deg)     # without the raw argmax
    ctx.sync_status()
    np.testing.assert_array_equal(r2["argmax_idx"].cpu().numpy(), r["argmax_idx"].cpu().numpy())
    np.testing.assert_array_equal(r2["smoothed"].cpu().numpy(), r["smoothed"].cpu().numpy())
    sm_ref, idx_ref, val_ref, ridx_ref, rval_ref = smooth.smooth_argmax(vals, g1, g2, bw, deg)
    sm = r["smoothed"].cpu().numpy().reshape(S, g1, g2)
    np.testing.assert_allclose(sm, sm_ref, rtol=0, atol=2e-6)
    gi = r["argmax_idx"].cpu().numpy()
    for s in range(S):
        # the GPU's argmax is a maximiser of the exact smoothed surface up to FP32 rounding
        assert sm_ref[s].ravel()[gi[s]] >= val_ref[s] - 4e-6
        assert r["argmax_val"][s].item() == pytest.approx(sm[s].ravel()[gi[s]], abs=0)
    np.testing.assert_array_equal(r["raw_idx"].cpu().numpy(), ridx_ref)
    np.testing.assert_array_equal(r["raw_val"].cpu().numpy(), rval_ref)


@pytest.mark.parametrize("shape,bw,deg", [((1, 101), 3.0, 2), ((64, 64), 3.0, 2), ((37, 150), 3.0, 2),
                                          ((5, 5), 3.0, 2), ((130, 9), 2.5, 1), ((1, 7), 4.0, 0),
                                          ((200, 1), 3.5, 2), ((33, 257), 2.5, 2)])
@pytest.mark.parametrize("offset", [0, 1])
def test_smoothing_f32_grid(ctx, shape, bw, deg, offset):
    """FP32 grids (mc_smooth_argmax_f32): on values that FP32 represents
    exactly, the outputs equal the FP64 entry point's bit for bit (both
    apply the stencil in FP32), and they match the oracle's least-squares
    fit of those values within the same 2e-6; offset 1 starts the input 4
    bytes past an 8-byte boundary (unpaired loads)."""
    import torch

    import paper_2005_10494_gb300 as pkg
    g1, g2 = shape
    S = 3
    rng = np.random.default_rng(g1 * 7 + g2)
    i, j = np.meshgrid(np.arange(g1), np.arange(g2), indexing="ij")
    vals = np.stack([0.7 - 0.0004 * (i - g1 / 3) ** 2 - 0.0002 * (j - g2 / 2) ** 2 + rng.normal(0, 0.01, (g1, g2))
                     for _ in range(S)]).astype(np.float32)
    base = torch.zeros(S * g1 * g2 + 1, dtype=torch.float32, device="cuda")
    v32 = base[offset:offset + S * g1 * g2]
    v32.copy_(torch.as_tensor(vals.ravel()))
    r32 = pkg.mc_smooth_argmax(ctx, v32, S, g1, g2, bandwidth=bw, degree=deg, raw=True)
    r64 = pkg.mc_smooth_argmax(ctx, v32.double(), S, g1, g2, bandwidth=bw, degree=deg, raw=True)
    ctx.sync_status()
    assert r32["smoothed"].dtype == torch.float32 and r32["argmax_val"].dtype == torch.float32
    np.testing.assert_array_equal(r32["smoothed"].double().cpu().numpy(), r64["smoothed"].cpu().numpy())
    for k in ("argmax_idx", "argmax_val", "raw_idx", "raw_val"):
        np.testing.assert_array_equal(r32[k].cpu().numpy().astype(np.float64), r64[k].cpu().numpy().astype(np.float64))
    sm_ref, idx_ref, val_ref, ridx_ref, rval_ref = smooth.smooth_argmax(vals.astype(np.float64), g1, g2, bw, deg)
    np.testing.assert_allclose(r32["smoothed"].cpu().numpy().reshape(S, g1, g2), sm_ref, rtol=0, atol=2e-6)
    np.testing.assert_array_equal(r32["raw_idx"].cpu().numpy(), ridx_ref)


# ------------------------------------------------------------ error paths
def test_error_paths(ctx):
    import torch

    import paper_2005_10494_gb300 as pkg
    from paper_2005_10494_gb300.binding import MCD_EINVAL, MCD_ENAN, MCD_ENOTSPD, MCD_EUNSUPPORTED
    bad = np.array([[1.0, 2.0], [2.0, 1.0]])
    prob = workloads.Problem("bad", [np.eye(2), bad], [0, 1, 1], [np.zeros(2)] * 3, [np.ones(2)] * 3,
                             [100, 100, 100], [0, 1, 2])
    dp = pkg.DeviceProblem.from_workload(prob)
    plan = pkg.Plan(ctx, dp)
    plan.eval(0)
    with pytest.raises(pkg.MCDError) as e:
        ctx.sync_status()
    assert e.value.code == MCD_ENOTSPD and e.value.index == 1
    ctx.sync_status()   # cleared
    mu = np.zeros(2)
    mu[1] = np.nan
    prob = workloads.Problem("nan", [np.eye(2)], [0, 0], [np.zeros(2), mu], [np.ones(2)] * 2, [100, 100], [0, 1])
    dp = pkg.DeviceProblem.from_workload(prob)
    pkg.Plan(ctx, dp).eval(0)
    with pytest.raises(pkg.MCDError) as e:
        ctx.sync_status()
    assert e.value.code == MCD_ENAN and e.value.index == 1
    S21 = torch.eye(21, dtype=torch.float64, device="cuda").reshape(-1)
    v = torch.zeros(21, dtype=torch.float64, device="cuda")
    dp = pkg.DeviceProblem([21], [0], [10], [0], S21, v, v)
    with pytest.raises(pkg.MCDError) as e:
        pkg.Plan(ctx, dp)
    assert e.value.code == MCD_EUNSUPPORTED
    dp = pkg.DeviceProblem.from_workload(workloads.c1(n_draws=10).subset([0]))
    dp.c.Sigma = np.zeros(9).ctypes.data       # host pointer
    with pytest.raises(pkg.MCDError) as e:
        pkg.Plan(ctx, dp)
    assert e.value.code == MCD_EINVAL
    dp = pkg.DeviceProblem.from_workload(workloads.c1(n_draws=10).subset([0]))
    with pytest.raises(pkg.MCDError):
        pkg.Plan(ctx, dp, grad=True, k=9)
    v = torch.zeros(100, dtype=torch.float64, device="cuda")
    with pytest.raises(pkg.MCDError):
        pkg.mc_smooth_argmax(ctx, v, 1, 10, 10, bandwidth=5.0)
    with pytest.raises(pkg.MCDError):
        pkg.mc_smooth_argmax(ctx, v, 1, 10, 10, bandwidth=3.0, degree=3)


def test_gradient_plan_draw_limit(ctx):
    """A gradient plan refuses a design whose draws would put more than 2^32
    draws into one of its 32 fixed-point batch slots (the sums could
    overflow); smaller designs, and forward plans of any size, are planned.
    Plans are created only (nothing is launched)."""
    import paper_2005_10494_gb300 as pkg
    from paper_2005_10494_gb300.binding import MCD_EINVAL
    base = workloads.c1(n_draws=10, keys="independent").subset([3, 50])
    for n, grad, ok in ((2 ** 38, True, False), (2 ** 36, True, True), (2 ** 38, False, True)):
        prob = base.subset([0, 1])
        prob.n_draws = np.array([1000, n], np.uint64)
        dp = pkg.DeviceProblem.from_workload(prob)
        if ok:
            pkg.Plan(ctx, dp, grad=grad).close()
        else:
            with pytest.raises(pkg.MCDError) as e:
                pkg.Plan(ctx, dp, grad=grad)
            assert e.value.code == MCD_EINVAL and e.value.index == 1
    ctx.sync_status()


def test_empty_problem(ctx):
    prob = workloads.Problem("empty", [np.eye(3)], [], [], [], [], [])
    out = run(ctx, prob, seed=0)
    assert out["hits"].shape == (0,)


def test_mixed_dimension_single_launch_equals_separate(ctx):
    prob = workloads.c3(n_scen=6, draws_range=(2e3, 3e4))
    mixed = run(ctx, prob, seed=2)
    sep = np.zeros(prob.n_design, np.int64)
    for d in sorted(set(prob.scen_d.tolist())):
        idx = [j for j in range(prob.n_design) if prob.d_of(j) == d]
        sep[idx] = run(ctx, prob.subset(idx), seed=2)["hits"]
    np.testing.assert_array_equal(mixed["hits"], sep)
    idx = list(range(0, prob.n_design, 7))
    assert_discordance(mixed["hits"], oracle_same_stream(prob, 2, idx), idx)


def test_smoothing_of_an_unaligned_input(ctx):
    # an input that starts 8 bytes past a 16-byte boundary takes the
    # single-double staging path even with an even row length; the result
    # must equal that of the aligned copy bit for bit
    import torch

    import paper_2005_10494_gb300 as pkg
    S, g1, g2 = 3, 70, 96
    rng = np.random.default_rng(12)
    vals = 0.6 + rng.normal(0, 0.02, (S, g1, g2))
    base = torch.zeros(S * g1 * g2 + 1, dtype=torch.float64, device="cuda")
    base[1:] = torch.as_tensor(vals.ravel(), dtype=torch.float64)
    off = base[1:]
    assert off.data_ptr() % 16 == 8
    aligned = off.clone()
    r1 = pkg.mc_smooth_argmax(ctx, off, S, g1, g2, bandwidth=3.0, degree=2, raw=True)
    r2 = pkg.mc_smooth_argmax(ctx, aligned, S, g1, g2, bandwidth=3.0, degree=2, raw=True)
    ctx.sync_status()
    for k in ("smoothed", "argmax_idx", "argmax_val", "raw_idx", "raw_val"):
        np.testing.assert_array_equal(r1[k].cpu().numpy(), r2[k].cpu().numpy())
    sm_ref = smooth.smooth_argmax(vals, g1, g2, 3.0, 2)[0]
    np.testing.assert_allclose(r1["smoothed"].cpu().numpy().reshape(S, g1, g2), sm_ref, rtol=0, atol=2e-6)


# ------------------------------------------------------------ pipe rates
def test_pipe_rates_are_plausible(ctx):
    """Instruction-class rates (ops per SM clock) lie within what one SM can
    issue: four schedulers x 32 lanes, and no class reads zero."""
    import paper_2005_10494_gb300 as pkg
    from paper_2005_10494_gb300.binding import MCD_EINVAL, PIPE_CLASSES
    rates = pkg.pipe_rates(ctx, iters=1024)
    assert set(rates) == set(PIPE_CLASSES)
    for name, r in rates.items():
        assert 1.0 <= r <= 128.0 * 1.02, (name, r, rates)
    # FP32 FMA runs on both halves of the FMA pipe; a mix of FMA and logic
    # instructions issues at least as fast as either alone.
    assert rates["ffma"] >= 60.0
    assert rates["mixed"] >= 0.95 * min(rates["ffma"], rates["lop3"])
    again = pkg.pipe_rates(ctx, iters=4096, classes=("ffma", "lg2"))
    for name in again:
        assert again[name] == pytest.approx(rates[name], rel=0.1)
    with pytest.raises(pkg.MCDError) as e:
        pkg.pipe_rates(ctx, iters=0, classes=("ffma",))
    assert e.value.code == MCD_EINVAL
