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
      argmax (the grid + smoothing route).

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
