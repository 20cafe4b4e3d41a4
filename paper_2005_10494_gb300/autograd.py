"""torch.autograd wrapper: p(mu, b) per design with the adjoint of the same
sampling pass (likelihood ratio, Appendix A.3 smoothness)."""
import torch

from .binding import MCD_ALL_BELOW


class MCDesignEval(torch.autograd.Function):
    """p = P(X_i > b_i for some i), X ~ N(mu, Sigma), for every design of a
    plan created with grad=True and k=0 whose problem's mu and b are the
    tensors passed here.  Backward: d p_j / d mu_j = Sigma^-1 E[(1_R - p)(X - mu)]
    (likelihood ratio with control variate), d p_j / d b_j = -d p_j / d mu_j.
    """

    @staticmethod
    def forward(ctx, mu, b, plan, seed):
        prob = plan.prob
        if mu.data_ptr() != prob.mu.data_ptr() or b.data_ptr() != prob.b.data_ptr():
            raise ValueError("mu and b must be the tensors the plan's problem was built on")
        if plan.k != 0:
            raise ValueError("MCDesignEval needs a plan with k = 0 (gradients in mu)")
        out = plan.grad(seed, None, 0.0)
        g = out["grad_lr"].clone()
        idx = torch.repeat_interleave(torch.arange(prob.n_design, device=mu.device),
                                      torch.as_tensor(prob.design_d, device=mu.device, dtype=torch.int64))
        ctx.save_for_backward(g, idx)
        return out["p"].clone()

    @staticmethod
    def backward(ctx, gp):
        g, idx = ctx.saved_tensors
        gm = gp[idx] * g
        return gm, -gm, None, None


def design_eval(mu, b, plan, seed):
    return MCDesignEval.apply(mu, b, plan, seed)


__all__ = ["MCDesignEval", "design_eval", "MCD_ALL_BELOW"]
