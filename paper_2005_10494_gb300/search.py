"""Design search driven by the adjoint, and the grid + smoothing alternative.

Sec. 2.1 solves the design problem by quasi-Newton steps on the objective;
Sec. 2.3 smooths Monte Carlo estimates over a grid and starts from the best
smoothed point because finite differences of noisy estimates mislead the
search.  With the adjoint of the sampling pass (likelihood-ratio estimate of
d p / d theta) the search can follow Monte Carlo gradients directly:

  gradient_search -- projected Adam ascent on p(q, a) over the box of cutoff
      quantiles q and allocations a, one mc_design_grad launch per step with
      a fixed stream key (common random numbers across steps);
  grid_argmax     -- mc_design_eval over the grid, local-quadratic smoothing,
      argmax (the grid + smoothing route);
  optimise_alpha  -- the paper's alpha optimisation for one set of nested
      populations (Sec. 2.1-2.3): N3 splits of the alpha budget, each scaled
      to the FWER constraint on the device (mc_fwer_calibrate), the expected
      power of each (Eq. 4, prior folded in) from shared draws, a thin-plate
      spline over the splits and its maximiser (mc_tps_fit / mc_tps_argmax);
  optimise_design -- the outer loop over nested populations r (Sec. 2.4):
      optimise_alpha for every r, a spline of the optimal power over r and
      its maximiser.

Both return the design parameters; evaluating them exactly is the caller's
business.  All sampling runs in libmcdesign; this module only loops.
"""
import numpy as np

from . import binding


def gradient_search(ctx, region_fn, Sigma, x0, lo, hi, n_draws, seed=0, key=0, steps=120, lr=0.02,
                    lr_final=0.002, betas=(0.9, 0.99), h=0.0):
    """Maximise p(x) over the box lo <= x <= hi.

    region_fn(x) -> (mu[d], b[d], jac[d][>=k]) gives the rejection region of
    the design with parameters x (k = len(x)) and the Jacobian of t = b - mu
    (its first k columns are used); Sigma is the d x d correlation matrix.
    Returns (x_best, p_best, history) where x_best is the final iterate and
    history holds (x, p_hat, grad) per step.
    """
    import torch
    x = np.asarray(x0, dtype=np.float64).copy()
    lo, hi = np.asarray(lo, np.float64), np.asarray(hi, np.float64)
    k = x.shape[0]
    mu, b, jac = region_fn(x)
    dev = torch.device("cuda", ctx.device)
    f64 = torch.float64
    d = len(mu)
    Sigma = torch.as_tensor(np.ascontiguousarray(Sigma), dtype=f64, device=dev).reshape(-1).contiguous()
    mu_t = torch.as_tensor(mu, dtype=f64, device=dev).contiguous()
    b_t = torch.as_tensor(b, dtype=f64, device=dev).contiguous()
    jac_t = torch.as_tensor(np.asarray(jac)[:, :k], dtype=f64, device=dev).reshape(-1).contiguous()
    prob = binding.DeviceProblem([d], [0], [n_draws], [key], Sigma, mu_t, b_t)
    plan = binding.Plan(ctx, prob, grad=True, k=k)
    m = np.zeros(k)
    v = np.zeros(k)
    hist = []
    for it in range(steps):
        mu, b, jac = region_fn(x)
        mu_t.copy_(torch.as_tensor(mu, dtype=f64))
        b_t.copy_(torch.as_tensor(b, dtype=f64))
        jac_t.copy_(torch.as_tensor(np.asarray(jac)[:, :k].reshape(-1), dtype=f64))
        out = plan.grad(seed, jac_t, h)
        g = out["grad_lr"].cpu().numpy()[:k].copy()
        p = float(out["p"].cpu().numpy()[0])
        hist.append((x.copy(), p, g.copy()))
        m = betas[0] * m + (1 - betas[0]) * g
        v = betas[1] * v + (1 - betas[1]) * g * g
        mh = m / (1 - betas[0] ** (it + 1))
        vh = v / (1 - betas[1] ** (it + 1))
        step_lr = lr * (lr_final / lr) ** (it / max(1, steps - 1))
        x = np.clip(x + step_lr * mh / (np.sqrt(vh) + 1e-12) * (hi - lo), lo, hi)
    ctx.sync_status()
    plan.close()
    return x, hist[-1][1], hist


def grid_argmax(ctx, prob, g1, g2, seed=0, bandwidth=3.0, degree=2):
    """mc_design_eval over a g1 x g2 grid of one scenario, then smoothing and
    argmax; returns (row index, column index, smoothed p at the argmax)."""
    dp = binding.DeviceProblem.from_workload(prob)
    plan = binding.Plan(ctx, dp)
    out = plan.eval(seed)
    r = binding.mc_smooth_argmax(ctx, out["p"], 1, g1, g2, bandwidth=bandwidth, degree=degree)
    ctx.sync_status()
    idx = int(r["argmax_idx"].item())
    plan.close()
    return idx // g2, idx % g2, float(r["argmax_val"].item())


def _dev(a, device):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), dtype=torch.float64, device=device)


def _alpha_estimates(ctx, cond, r, n3, n_draws, seed, rounds, u=None):
    """The noisy expected power of the N3 alpha splits of one r (the first
    half of optimise_alpha): box points u, each split's scale calibrated to
    the FWER on the device (n_draws per round, one stream for all splits),
    then its power under the prior-folded alternative (n_draws, one stream).
    Returns u (host), the points x (device, [1][N3][n-1]), p_hat (device)
    and the plan, which the caller closes once the queued work is done."""
    import torch

    import workloads
    n = r.shape[0]
    m, C, Sig0 = workloads.paper_law(cond, r)
    if u is None:
        u = workloads.box_points(n3, n - 1, seed)
    w = workloads.split_from_box(u)
    N3 = w.shape[0]
    dev = torch.device("cuda", ctx.device)
    zeros = _dev(np.zeros(N3 * n), dev)
    null = binding.DeviceProblem([n], np.zeros(N3), np.full(N3, n_draws), np.zeros(N3), _dev(Sig0.ravel(), dev),
                                 zeros, zeros)
    cal = binding.mc_fwer_calibrate(ctx, null, _dev(w.ravel(), dev), workloads.ALPHA0, rounds=rounds, seed=seed)
    alt = binding.DeviceProblem([n], np.zeros(N3), np.full(N3, n_draws), np.ones(N3), _dev(C.ravel(), dev),
                                _dev(np.tile(m, N3), dev), cal["b"])
    plan = binding.Plan(ctx, alt, shared=True)
    p_hat = plan.eval(seed + 1)["p"]
    return u, _dev(u, dev).reshape(1, N3, n - 1), p_hat, plan


def optimise_alpha(ctx, cond, r, n3=2000, n_draws=10_000_000, seed=0, smoothing=1e-6, rounds=8,
                   final_draws=100_000_000, u=None):
    """Maximise the expected power over the alpha allocations of condition
    `cond` (workloads.PAPER_EFFECTS) at population fractions r, with the
    FWER constraint of Eq. 2 (alpha0 = 0.025).

    Points u of the box [0,1]^(n-1) map to splits w (workloads.split_from_box);
    each split's scale is calibrated on the device under the null
    (n_draws per round, one stream for all splits), its expected power
    estimated under the prior-folded alternative (n_draws, one stream for all
    splits), a thin-plate spline with `smoothing` (a value, or "gcv": the
    minimiser of the GCV score over 1e-10 .. 1e-2) is fitted over u and
    maximised in the box, and the split at the maximiser is calibrated once
    more with final_draws (skipped when final_draws is 0: alpha and scale
    are then None).  Eight calibration rounds leave |FWER - alpha0|
    at the returned scale near 1e-6, a few per cent of the estimate's own
    Monte Carlo error at 1e7 draws; 14 rounds give the same scales to four
    digits.  Returns dict u, alpha, p_fit (the spline's maximum), p_hat
    (the point estimates), scale, smoothing."""
    import torch

    import workloads
    r = np.asarray(r, dtype=np.float64)
    n = r.shape[0]
    dev = torch.device("cuda", ctx.device)
    u, x, p_hat, plan = _alpha_estimates(ctx, cond, r, n3, n_draws, seed, rounds, u)
    N3 = u.shape[0]
    Sig0 = workloads.paper_law(cond, r)[2]
    if isinstance(smoothing, str):
        grid = np.logspace(-10, -2, 17)
        score = binding.mc_tps_gcv(ctx, x[0], p_hat, grid).cpu().numpy()
        smoothing = float(grid[int(np.nanargmin(score))])
    fit = binding.mc_tps_fit(ctx, x, p_hat.reshape(1, N3), smoothing=smoothing)
    lo, hi = _dev(np.zeros(n - 1), dev), _dev(np.ones(n - 1), dev)
    am = binding.mc_tps_argmax(ctx, x, fit, lo, hi, iters=300)
    ctx.sync_status()
    u_star = am["x"].cpu().numpy()[0]
    w_star = workloads.split_from_box(u_star)[0]
    plan.close()
    if not final_draws:
        # the caller needs only the spline's maximum (the loop over r)
        return {"u": u_star, "alpha": None, "scale": None, "p_fit": float(am["f"].item()),
                "p_hat": p_hat.cpu().numpy(), "smoothing": smoothing}
    one = binding.DeviceProblem([n], [0], [final_draws], [2], _dev(Sig0.ravel(), dev), _dev(np.zeros(n), dev),
                                _dev(np.zeros(n), dev))
    c1 = binding.mc_fwer_calibrate(ctx, one, _dev(w_star, dev), workloads.ALPHA0, rounds=rounds, seed=seed + 2)
    ctx.sync_status()
    scale = float(c1["scale"].item())
    return {"u": u_star, "alpha": scale * w_star, "scale": scale, "p_fit": float(am["f"].item()),
            "p_hat": p_hat.cpu().numpy(), "smoothing": smoothing}


def r_search_box(per_r):
    """Spline coordinates and search box of the choice of r (host only).

    per_r: list of (r2, r3, optimal power).  Returns the points (r2, r3/r2),
    their values, and the box lo, hi: within two grid steps of the best
    pair, inside the range of the evaluated points, and with r3 = r2 * (r3/r2)
    at or above the smallest evaluated r3 (a rectangle in these coordinates
    would otherwise reach below it at small r2 with the smallest ratio,
    where the spline has no data)."""
    pts = np.array([[a, b / a] for a, b, _ in per_r])
    vals = np.array([v for _, _, v in per_r])
    ib = int(np.argmax(vals))
    step = float(np.min(np.diff(np.unique(pts[:, 0])))) if len(np.unique(pts[:, 0])) > 1 else 0.05
    reach = np.array([2.0 * step, 2.0 * step / pts[ib, 0]])
    lo = np.maximum(pts.min(0), pts[ib] - reach)
    hi = np.minimum(pts.max(0), pts[ib] + reach)
    r3_min = min(b for _, b, _ in per_r)
    lo[1] = min(max(lo[1], r3_min / lo[0]), hi[1])
    return pts, vals, lo, hi


def optimise_design(ctx, cond, r_pairs=None, n3=2000, n_draws=10_000_000, seed=0, smoothing=1e-6,
                    r_smoothing=1e-6):
    """The choice of nested populations for n = 3 (Sec. 2.4 with power as
    the utility): optimise_alpha at every r = (1, r2, r3) of r_pairs
    (default the paper's 171 pairs), a thin-plate spline of the optimal power
    over (r2, r3 / r2), its maximiser within two grid steps of the best
    evaluated pair (the search starts from the best point, as Sec. 2.3 does
    for alpha; the box stays inside the range of the evaluated pairs and
    keeps r3 at or above the smallest evaluated r3, so 1 > r2 > r3 > 0 holds
    and the spline is not extrapolated into regions without data), and
    optimise_alpha at the maximiser.  Returns dict r,
    alpha, p_fit, per_r (list of (r2, r3, p_fit))."""
    import torch

    import workloads
    pairs = workloads.paper_r_pairs() if r_pairs is None else r_pairs
    per_r = []
    if isinstance(smoothing, str):
        for q, (r2, r3) in enumerate(pairs):
            res = optimise_alpha(ctx, cond, (1.0, r2, r3), n3=n3, n_draws=n_draws, seed=seed + 7 * q,
                                 smoothing=smoothing, final_draws=0)
            per_r.append((r2, r3, res["p_fit"]))
    else:
        # the same per-pair estimates as optimise_alpha, then the splines of
        # all pairs fitted in one call (independent fits run concurrently)
        # and maximised in one call (one cluster per surface)
        xs, ps, plans = [], [], []
        for q, (r2, r3) in enumerate(pairs):
            _, xq, pq, plq = _alpha_estimates(ctx, cond, np.array([1.0, r2, r3]), n3, n_draws, seed + 7 * q, 8)
            xs.append(xq[0])
            ps.append(pq)
            plans.append(plq)
        dev0 = torch.device("cuda", ctx.device)
        xa = torch.stack(xs)
        fits = binding.mc_tps_fit(ctx, xa, torch.stack(ps), smoothing=smoothing)
        k = xa.shape[2]
        am = binding.mc_tps_argmax(ctx, xa, fits, _dev(np.zeros(k), dev0), _dev(np.ones(k), dev0), iters=300)
        ctx.sync_status()
        for plq in plans:
            plq.close()
        f = am["f"].cpu().numpy()
        per_r = [(r2, r3, float(f[q])) for q, (r2, r3) in enumerate(pairs)]
    dev = torch.device("cuda", ctx.device)
    pts, vals, lo_np, hi_np = r_search_box(per_r)
    x = _dev(pts, dev).reshape(1, len(per_r), 2)
    fit = binding.mc_tps_fit(ctx, x, _dev(vals, dev).reshape(1, -1), smoothing=r_smoothing)
    lo, hi = _dev(lo_np, dev), _dev(hi_np, dev)
    am = binding.mc_tps_argmax(ctx, x, fit, lo, hi, iters=300)
    ctx.sync_status()
    r2s, v = am["x"].cpu().numpy()[0]
    r_best = (1.0, float(r2s), float(r2s * v))
    best = optimise_alpha(ctx, cond, r_best, n3=n3, n_draws=n_draws, seed=seed + 1000, smoothing=smoothing)
    return {"r": r_best, "alpha": best["alpha"], "p_fit": best["p_fit"], "per_r": per_r}
