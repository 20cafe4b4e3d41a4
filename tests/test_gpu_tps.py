"""Thin-plate spline fit and maximiser on the device (Sec. 2.3) against the
FP64 oracle: fitted values and the fitted function at query points, the
maximiser in a box, several surfaces per call, the paper-size case, error
paths."""
import numpy as np
import pytest

from oracle import tps

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2005_10494_gb300 as pkg
    return pkg.Context(0)


def data(rng, n, k, noise=0.05):
    x = rng.uniform(0, 1, (n, k))
    y = np.exp(-3.0 * ((x - 0.55) ** 2).sum(1)) + rng.normal(0, noise, n)
    return x, y


def gpu_fit(ctx, xs, ys, s):
    import torch

    import paper_2005_10494_gb300 as pkg
    xt = torch.as_tensor(np.stack(xs), dtype=torch.float64, device="cuda")
    yt = torch.as_tensor(np.stack(ys), dtype=torch.float64, device="cuda")
    out = pkg.mc_tps_fit(ctx, xt, yt, smoothing=s)
    ctx.sync_status()
    return xt, out


@pytest.mark.parametrize("k,n,s", [(1, 150, 1e-3), (1, 97, 0.5), (2, 300, 0.0), (2, 257, 0.05), (2, 513, 2.0),
                                   (3, 257, 0.0), (3, 200, 0.3)])
def test_fit_matches_oracle(ctx, k, n, s):
    rng = np.random.default_rng(100 * k + n)
    x, y = data(rng, n, k)
    _, out = gpu_fit(ctx, [x], [y], s)
    coef = out["coef"].cpu().numpy()[0]
    c_ref, d_ref = tps.fit(x, y, s)
    fit_ref = tps.evaluate(x, x, c_ref, d_ref)
    np.testing.assert_allclose(out["fitted"].cpu().numpy()[0], fit_ref, rtol=0, atol=1e-8)
    xq = rng.uniform(0, 1, (64, k))
    np.testing.assert_allclose(tps.evaluate(xq, x, coef[:n], coef[n:]), tps.evaluate(xq, x, c_ref, d_ref),
                               rtol=0, atol=1e-8)
    # side conditions of the spline
    np.testing.assert_allclose(np.hstack([np.ones((n, 1)), x]).T @ coef[:n], 0.0, atol=1e-8)


@pytest.mark.parametrize("n", [1, 5, 31, 32, 33, 64, 65, 97])
def test_fit_at_block_edges(ctx, n):
    """The projected system has n = n_pts - k - 1 rows, factored in blocks of
    32 with one block of look-ahead and solved one block per launch: one
    block only (n <= 32), a last block of one row (33, 65), exact multiples."""
    k = 2
    rng = np.random.default_rng(700 + n)
    x, y = data(rng, n + k + 1, k)
    _, out = gpu_fit(ctx, [x], [y], 0.05)
    c_ref, d_ref = tps.fit(x, y, 0.05)
    np.testing.assert_allclose(out["fitted"].cpu().numpy()[0], tps.evaluate(x, x, c_ref, d_ref), rtol=0, atol=1e-8)


def test_several_surfaces_and_paper_size(ctx):
    rng = np.random.default_rng(5)
    xs, ys = [], []
    for _ in range(3):
        x, y = data(rng, 2000, 2, noise=0.01)
        xs.append(x)
        ys.append(y)
    _, out = gpu_fit(ctx, xs, ys, 0.01)
    for q in range(3):
        c_ref, d_ref = tps.fit(xs[q], ys[q], 0.01)
        np.testing.assert_allclose(out["fitted"].cpu().numpy()[q], tps.evaluate(xs[q], xs[q], c_ref, d_ref),
                                   rtol=0, atol=1e-8)


def test_many_surfaces_on_worker_streams(ctx):
    """Nine surfaces in one call: up to four worker streams fit two or three
    surfaces each in turn, each surface against its own oracle fit."""
    rng = np.random.default_rng(91)
    xs, ys = [], []
    for q in range(9):
        x, y = data(rng, 180 + 7 * q, 2, noise=0.02)
        xs.append(x[:180])
        ys.append(y[:180])
    _, out = gpu_fit(ctx, xs, ys, 0.02)
    fitted = out["fitted"].cpu().numpy()
    for q in range(9):
        c_ref, d_ref = tps.fit(xs[q], ys[q], 0.02)
        np.testing.assert_allclose(fitted[q], tps.evaluate(xs[q], xs[q], c_ref, d_ref), rtol=0, atol=1e-8)


def test_grid_of_4096_points(ctx):
    # the 64 x 64 design grid of one scenario as scattered points
    g = np.linspace(0.05, 0.95, 64)
    qq, aa = np.meshgrid(g, np.linspace(0.2, 0.8, 64), indexing="ij")
    x = np.stack([qq.ravel(), aa.ravel()], 1)
    rng = np.random.default_rng(9)
    y = 0.9 - (qq.ravel() - 0.6) ** 2 - 0.5 * (aa.ravel() - 0.5) ** 2 + rng.normal(0, 1e-3, x.shape[0])
    _, out = gpu_fit(ctx, [x], [y], 1e-4)
    c_ref, d_ref = tps.fit(x, y, 1e-4)
    np.testing.assert_allclose(out["fitted"].cpu().numpy()[0], tps.evaluate(x, x, c_ref, d_ref), rtol=0, atol=1e-8)


@pytest.mark.parametrize("k", [1, 2, 3])
def test_argmax_matches_oracle(ctx, k):
    import torch

    import paper_2005_10494_gb300 as pkg
    rng = np.random.default_rng(20 + k)
    x, y = data(rng, 300, k, noise=0.02)
    s = 0.05
    xt, out = gpu_fit(ctx, [x], [y], s)
    lo = torch.full((k,), 0.0, dtype=torch.float64, device="cuda")
    hi = torch.full((k,), 1.0, dtype=torch.float64, device="cuda")
    res = pkg.mc_tps_argmax(ctx, xt, out, lo, hi, iters=300)
    ctx.sync_status()
    xg, fg = res["x"].cpu().numpy()[0], float(res["f"].cpu().numpy()[0])
    c_ref, d_ref = tps.fit(x, y, s)
    xr, fr = tps.argmax(x, c_ref, d_ref, np.zeros(k), np.ones(k))
    assert fg == pytest.approx(fr, abs=1e-9)
    np.testing.assert_allclose(xg, xr, atol=2e-4)
    assert fg == pytest.approx(tps.evaluate(xg, x, c_ref, d_ref)[0], abs=1e-9)
    # an interior maximiser: the gradient vanishes there
    if np.all((xg > 1e-6) & (xg < 1 - 1e-6)):
        assert np.max(np.abs(tps.gradient(xg, x, c_ref, d_ref))) < 1e-5


def test_argmax_of_several_surfaces(ctx):
    """Each surface is maximised by its own thread-block cluster: four
    surfaces of different peaks in one call, each against the oracle's
    maximiser of its own fit."""
    import torch

    import paper_2005_10494_gb300 as pkg
    rng = np.random.default_rng(77)
    xs, ys, peaks = [], [], [(0.3, 0.7), (0.6, 0.4), (0.5, 0.5), (0.8, 0.2)]
    for pk in peaks:
        x = rng.uniform(0, 1, (250, 2))
        y = np.exp(-4.0 * ((x - np.array(pk)) ** 2).sum(1)) + rng.normal(0, 0.01, 250)
        xs.append(x)
        ys.append(y)
    xt, out = gpu_fit(ctx, xs, ys, 0.05)
    lo = torch.zeros(2, dtype=torch.float64, device="cuda")
    hi = torch.ones(2, dtype=torch.float64, device="cuda")
    res = pkg.mc_tps_argmax(ctx, xt, out, lo, hi, iters=300)
    ctx.sync_status()
    xg, fg = res["x"].cpu().numpy(), res["f"].cpu().numpy()
    for q in range(len(peaks)):
        c_ref, d_ref = tps.fit(xs[q], ys[q], 0.05)
        xr, fr = tps.argmax(xs[q], c_ref, d_ref, np.zeros(2), np.ones(2))
        assert fg[q] == pytest.approx(fr, abs=1e-9)
        np.testing.assert_allclose(xg[q], xr, atol=2e-4)


def test_argmax_on_the_box_boundary(ctx):
    import torch

    import paper_2005_10494_gb300 as pkg
    rng = np.random.default_rng(31)
    x = rng.uniform(0, 1, (200, 2))
    y = 0.5 + 0.3 * x[:, 0] - 0.2 * (x[:, 1] - 0.4) ** 2 + rng.normal(0, 0.01, 200)   # increasing in x0
    xt, out = gpu_fit(ctx, [x], [y], 0.1)
    lo = torch.tensor([0.0, 0.0], dtype=torch.float64, device="cuda")
    hi = torch.tensor([0.8, 1.0], dtype=torch.float64, device="cuda")
    res = pkg.mc_tps_argmax(ctx, xt, out, lo, hi, iters=300)
    xg = res["x"].cpu().numpy()[0]
    c_ref, d_ref = tps.fit(x, y, 0.1)
    xr, fr = tps.argmax(x, c_ref, d_ref, np.array([0.0, 0.0]), np.array([0.8, 1.0]))
    assert xg[0] == pytest.approx(0.8, abs=1e-12)
    np.testing.assert_allclose(xg, xr, atol=2e-4)
    assert float(res["f"].item()) == pytest.approx(fr, abs=1e-9)


def test_repeated_points_and_bad_arguments(ctx):
    import torch

    import paper_2005_10494_gb300 as pkg
    from paper_2005_10494_gb300.binding import MCD_EINVAL, MCD_ENOTSPD
    rng = np.random.default_rng(2)
    x, y = data(rng, 50, 2)
    x2 = x.copy()
    x2[7] = x2[3]                                    # a repeated point: singular without smoothing
    xt = torch.as_tensor(np.stack([x, x2]), dtype=torch.float64, device="cuda")
    yt = torch.as_tensor(np.stack([y, y]), dtype=torch.float64, device="cuda")
    out = pkg.mc_tps_fit(ctx, xt, yt, smoothing=0.0)
    with pytest.raises(pkg.MCDError) as e:
        ctx.sync_status()
    assert e.value.code == MCD_ENOTSPD and e.value.index == 1
    c = out["coef"].cpu().numpy()
    assert np.all(np.isfinite(c[0])) and np.all(np.isnan(c[1]))
    out = pkg.mc_tps_fit(ctx, xt, yt, smoothing=0.1)      # smoothing makes it definite again
    ctx.sync_status()
    assert np.all(np.isfinite(out["coef"].cpu().numpy()))
    for kw in ({"smoothing": -1.0}, {"smoothing": float("inf")}):
        with pytest.raises(pkg.MCDError) as e:
            pkg.mc_tps_fit(ctx, xt, yt, **kw)
        assert e.value.code == MCD_EINVAL
    with pytest.raises(pkg.MCDError) as e:
        pkg.mc_tps_fit(ctx, xt[:, :3], yt[:, :3])            # n_pts < k + 2
    assert e.value.code == MCD_EINVAL


@pytest.mark.parametrize("k,n,lo", [(2, 300, -6), (1, 97, -4), (3, 130, -5), (2, 65, -6), (2, 36, -5)])
def test_gcv_matches_oracle(ctx, k, n, lo):
    import torch

    import paper_2005_10494_gb300 as pkg
    rng = np.random.default_rng(70 + k + n)
    x, y = data(rng, n, k)
    s_values = np.logspace(lo, 0.5, 7)
    xt = torch.as_tensor(x, dtype=torch.float64, device="cuda")
    yt = torch.as_tensor(y, dtype=torch.float64, device="cuda")
    gpu = pkg.mc_tps_gcv(ctx, xt, yt, s_values).cpu().numpy()
    ctx.sync_status()
    ref = np.array([tps.gcv(x, y, s) for s in s_values])
    np.testing.assert_allclose(gpu, ref, rtol=1e-7)
    assert int(np.argmin(gpu)) == int(np.argmin(ref))


def test_gcv_rejects_bad_values(ctx):
    import torch

    import paper_2005_10494_gb300 as pkg
    from paper_2005_10494_gb300.binding import MCD_EINVAL
    x = torch.rand(50, 2, dtype=torch.float64, device="cuda")
    y = torch.rand(50, dtype=torch.float64, device="cuda")
    for bad in ([0.0], [1.0, -1.0], [float("inf")], []):
        with pytest.raises(pkg.MCDError) as e:
            pkg.mc_tps_gcv(ctx, x, y, bad)
        assert e.value.code == MCD_EINVAL
