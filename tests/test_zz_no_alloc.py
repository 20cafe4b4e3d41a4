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
