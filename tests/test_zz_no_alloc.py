"""The allocation-free entry point against the planned one.

mc_design_eval_noalloc serves callers that cannot allocate device memory
where they evaluate designs (their own up-front memory pools, loops that must
not synchronise on cudaMalloc / cudaFree).  Its scratch is a static device
array shared by all calls, so two calls in a row must each give exactly what
mc_design_eval gives: hit counts are integers and must match bit for bit, p
and se follow from them by the same FP64 formula.
"""
import ctypes

import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu


def _problems():
    rng = np.random.default_rng(21)
    S = workloads.lkj_cvine(7, 2.0, rng)
    mus = [rng.normal(0.3, 0.4, 7) for _ in range(40)]
    bs = [np.full(7, 2.2) for _ in range(40)]
    lkj7 = workloads.Problem("lkj7", [S], [0] * 40, mus, bs, [123_457] * 40, rng.integers(0, 2**40, 40))
    return [workloads.c1(n_draws=100_000, keys="independent"),
            workloads.c4(g1=4, g2=4, n_draws=300_001, keys="independent"),
            lkj7]


def test_noalloc_matches_mc_design_eval_on_two_calls():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2005_10494_gb300 as pkg
    lib = pkg.load()
    ctx = pkg.Context(0)
    for prob in _problems():
        dp = pkg.DeviceProblem.from_workload(prob)
        J = prob.n_design
        hits = torch.empty(J, dtype=torch.int64, device="cuda")
        p = torch.empty(J, dtype=torch.float64, device="cuda")
        se = torch.empty(J, dtype=torch.float64, device="cuda")
        stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        for seed in (11, 12):                      # two calls in a row share the scratch
            ref = pkg.mc_design_eval(ctx, dp, seed)
            ctx.sync_status()
            rc = lib.mc_design_eval_noalloc(0, ctypes.byref(dp.c), seed, ctypes.c_void_p(hits.data_ptr()),
                                            ctypes.c_void_p(p.data_ptr()), ctypes.c_void_p(se.data_ptr()), stream)
            assert rc == 0
            torch.cuda.synchronize()
            np.testing.assert_array_equal(hits.cpu().numpy(), ref["hits"].cpu().numpy())
            np.testing.assert_array_equal(p.cpu().numpy(), ref["p"].cpu().numpy())
            np.testing.assert_array_equal(se.cpu().numpy(), ref["se"].cpu().numpy())


def test_noalloc_rejects_what_its_scratch_cannot_hold():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2005_10494_gb300 as pkg
    lib = pkg.load()
    two = workloads.c2(n_scen=2, g1=2, g2=2, n_draws=1000)          # two scenarios
    dp = pkg.DeviceProblem.from_workload(two)
    assert lib.mc_design_eval_noalloc(0, ctypes.byref(dp.c), 0, None, None, None, None) == 1
    big = workloads.c2(n_scen=1, g1=130, g2=130, n_draws=10)       # 16900 > 16384 designs
    dp = pkg.DeviceProblem.from_workload(big)
    assert lib.mc_design_eval_noalloc(0, ctypes.byref(dp.c), 0, None, None, None, None) == 1


def _noalloc(lib, dp, seed):
    import torch
    J = dp.n_design
    hits = torch.full((J,), -1, dtype=torch.int64, device="cuda")
    p = torch.empty(J, dtype=torch.float64, device="cuda")
    se = torch.empty(J, dtype=torch.float64, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib.mc_design_eval_noalloc(0, ctypes.byref(dp.c), seed, ctypes.c_void_p(hits.data_ptr()),
                                    ctypes.c_void_p(p.data_ptr()), ctypes.c_void_p(se.data_ptr()), stream)
    assert rc == 0
    torch.cuda.synchronize()
    return hits.cpu().numpy(), p.cpu().numpy(), se.cpu().numpy()


def test_noalloc_documented_error_outputs():
    """The outputs the header documents for bad values in valid memory (no
    fault is involved): the complement region gives N - hits; a Sigma that is
    not positive definite gives p = se = NaN and hits = 0 for every design; a
    NaN in one design's mu or b gives that for the design alone, while the
    other designs keep the counts of mc_design_eval."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2005_10494_gb300 as pkg
    from paper_2005_10494_gb300.binding import MCD_ALL_BELOW, MCD_ENAN
    lib = pkg.load()
    ctx = pkg.Context(0)
    prob = workloads.c4(g1=3, g2=3, n_draws=200_003, keys="independent")
    N = 200_003

    dp = pkg.DeviceProblem.from_workload(prob)
    h_any, _, _ = _noalloc(lib, dp, 5)
    ref = pkg.mc_design_eval(ctx, dp, 5)
    ctx.sync_status()
    np.testing.assert_array_equal(h_any, ref["hits"].cpu().numpy())
    below = pkg.DeviceProblem.from_workload(prob, region=MCD_ALL_BELOW)
    h_below, p_below, se_below = _noalloc(lib, below, 5)
    np.testing.assert_array_equal(h_below, N - h_any)
    np.testing.assert_array_equal(p_below, 1.0 - h_any / N)
    np.testing.assert_allclose(se_below, np.sqrt(p_below * (1 - p_below) / N), rtol=1e-12, atol=0)

    # not positive definite: equicorrelation -0.2 in 10 dimensions has the
    # eigenvalue 1 + 9 (-0.2) < 0
    bad = workloads.equicorrelated(10, -0.2)
    assert np.linalg.eigvalsh(bad).min() < 0
    nonspd = workloads.Problem("nonspd", [bad], prob.design_scen, prob.mus, prob.bs, prob.n_draws, prob.keys)
    h, p, se = _noalloc(lib, pkg.DeviceProblem.from_workload(nonspd), 5)
    assert np.all(h == 0) and np.all(np.isnan(p)) and np.all(np.isnan(se))

    # a NaN in design 4's mu and one in design 7's b
    mus = [m.copy() for m in prob.mus]
    bs = [b.copy() for b in prob.bs]
    mus[4][3] = np.nan
    bs[7][9] = np.nan
    nanp = workloads.Problem("nan", prob.sigmas, prob.design_scen, mus, bs, prob.n_draws, prob.keys)
    dpn = pkg.DeviceProblem.from_workload(nanp)
    h, p, se = _noalloc(lib, dpn, 5)
    for j in (4, 7):
        assert h[j] == 0 and np.isnan(p[j]) and np.isnan(se[j])
    others = [j for j in range(prob.n_design) if j not in (4, 7)]
    np.testing.assert_array_equal(h[others], h_any[others])
    pkg.mc_design_eval(ctx, dpn, 5)
    with pytest.raises(pkg.MCDError) as e:          # the planned call reports it through the status word
        ctx.sync_status()
    assert e.value.code == MCD_ENAN and e.value.index in (4, 7)
    # the scratch keeps no state that a later good call could see
    h2, _, _ = _noalloc(lib, dp, 5)
    np.testing.assert_array_equal(h2, h_any)
