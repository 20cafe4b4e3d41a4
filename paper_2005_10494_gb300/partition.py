"""Sharding a batch of designs over ranks (one process per GPU).

Designs are independent Monte Carlo problems, so a batch splits over ranks
with no exchange during sampling: each rank evaluates a contiguous range of
designs, and the exact integer hit counts (and any per-design output) are
gathered afterwards.  Ranges are balanced by the sampling cost of a design,
which grows as N_j d_j^2 (N_j draws, each with a d_j x d_j triangular
transform; the generator's share, linear in d_j, is folded into the same
proxy).

  design_ranges -- contiguous [lo, hi) per rank with balanced cost;
  shard_problem -- the sub-problem of one rank (a workloads.Problem subset);
  gather_designs -- concatenate per-rank per-design arrays in design order
                    (torch.distributed all_gather of fixed-size buffers).

Host logic only: the sampling itself runs in libmcdesign on each rank's GPU.
"""
import numpy as np


def design_cost(n_draws, d):
    """Sampling cost proxy of each design: N_j * d_j^2."""
    return np.asarray(n_draws, dtype=np.float64) * np.asarray(d, dtype=np.float64) ** 2


def design_ranges(cost, world):
    """Split designs 0..J-1 into `world` contiguous ranges [lo, hi) whose
    summed cost is as even as a contiguous split allows: rank r's range ends
    at the first design whose cumulative cost reaches (r + 1)/world of the
    total.  Every design lands in exactly one range; ranges may be empty
    when there are fewer designs than ranks."""
    cost = np.asarray(cost, dtype=np.float64)
    if world < 1:
        raise ValueError("world must be >= 1")
    if np.any(cost < 0) or not np.all(np.isfinite(cost)):
        raise ValueError("costs must be finite and >= 0")
    J = cost.shape[0]
    csum = np.cumsum(cost)
    total = csum[-1] if J else 0.0
    bounds = [0]
    for r in range(1, world):
        if total > 0:
            # first index whose cumulative cost reaches the target
            cut = int(np.searchsorted(csum, total * r / world, side="left")) + 1
        else:
            cut = (J * r) // world
        bounds.append(min(J, max(bounds[-1], cut)))
    bounds.append(J)
    return [(bounds[r], bounds[r + 1]) for r in range(world)]


def shard_problem(prob, world, rank):
    """The designs of `rank`: (lo, hi, workloads.Problem of designs lo..hi-1)."""
    cost = design_cost(prob.n_draws, [prob.d_of(j) for j in range(prob.n_design)])
    lo, hi = design_ranges(cost, world)[rank]
    return lo, hi, prob.subset(range(lo, hi), name="%s-rank%d" % (prob.name, rank))


def gather_designs(local, ranges, group=None):
    """All-gather per-design values (a 1-D torch tensor per rank, the rank's
    range in design order) into the full array on every rank.  Buffers are
    padded to the longest range so that the collective sees equal shapes;
    the padding is dropped again.  Integer hit counts come back exactly."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    if len(ranges) != world:
        raise ValueError("one range per rank")
    longest = max(hi - lo for lo, hi in ranges)
    buf = torch.zeros(max(longest, 1), dtype=local.dtype, device=local.device)
    buf[:local.numel()] = local
    parts = [torch.empty_like(buf) for _ in range(world)]
    dist.all_gather(parts, buf, group=group)
    return torch.cat([parts[r][:hi - lo] for r, (lo, hi) in enumerate(ranges)])
