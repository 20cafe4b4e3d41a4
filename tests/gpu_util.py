"""Helpers for the GPU parity tests: run the CUDA path through the C ABI and
the FP64 oracle on the same seeded inputs."""
import math

import numpy as np

# Same-stream comparison radius (units of X).  The FP32 path forms z with
# approximate log2 / sqrt / sin / cos (errors below ~1e-5 for |z| <= 5.8) and
# y = L z with FP32 FMAs; |y_fp32 - y_exact| stays below ~6e-5 for d <= 20,
# so a draw's indicator can differ from the FP64 oracle's only if some
# |y_i - t_i| < EPS32.
EPS32 = 1e-4
# The FP64 path differs from the oracle only by the last bits of log / sin / cos.
EPS64 = 1e-9


def run(ctx, prob, seed=0, grad=False, k=0, jac=None, h=0.0, region=0, **plan_kw):
    import torch

    import paper_2005_10494_gb300 as pkg
    dp = pkg.DeviceProblem.from_workload(prob, region=region)
    plan = pkg.Plan(ctx, dp, grad=grad, k=k, **plan_kw)
    jt = None if jac is None else torch.as_tensor(jac, dtype=torch.float64, device="cuda")
    # graph replay needs a capturable (non-default) stream
    stream = torch.cuda.Stream() if plan_kw.get("graph") else None
    if stream is not None:
        stream.wait_stream(torch.cuda.current_stream())
    out = plan.grad(seed, jt, h, stream=stream) if grad else plan.eval(seed, stream=stream)
    if stream is not None:
        out = plan.grad(seed, jt, h, stream=stream) if grad else plan.eval(seed, stream=stream)  # replay
        stream.synchronize()
    ctx.sync_status()
    res = {name: t.cpu().numpy() for name, t in out.items()}
    plan.close()
    return res


def oracle_designs(prob, idx):
    return [{"Sigma": prob.sigmas[prob.design_scen[j]], "t": prob.t(j), "key": int(prob.keys[j]),
             "n_draws": int(prob.n_draws[j]), "draw_begin": int(prob.draw_begin[j])} for j in idx]


def oracle_same_stream(prob, seed, idx, eps=EPS32, grad=False, h=0.0):
    from oracle import mc
    return mc.mc_batch(oracle_designs(prob, idx), seed, eps=eps, grad=grad, h=h)


def report(name, **stats):
    """Append one JSON line of parity statistics (with the per-design records
    of the check) to the file named by the environment variable
    MCD_PARITY_REPORT (nothing when it is unset)."""
    import json
    import os
    path = os.environ.get("MCD_PARITY_REPORT")
    if path:
        with open(path, "a") as f:
            f.write(json.dumps(dict(check=name, **stats)) + "\n")


def assert_discordance(gpu_hits, ora, idx):
    """|hits_gpu - hits_oracle| <= ambiguous draws, design by design.
    Returns the number of designs, the total |difference| and ambiguous
    draws, and per design its counts."""
    bad, rec = [], []
    tot_diff = tot_amb = 0
    for k, j in enumerate(idx):
        diff = abs(int(gpu_hits[j]) - int(ora["hits"][k]))
        tot_diff += diff
        tot_amb += int(ora["ambiguous"][k])
        rec.append({"design": int(j), "hits_gpu": int(gpu_hits[j]), "hits_oracle": int(ora["hits"][k]),
                    "ambiguous": int(ora["ambiguous"][k])})
        if diff > int(ora["ambiguous"][k]):
            bad.append((j, int(gpu_hits[j]), int(ora["hits"][k]), int(ora["ambiguous"][k])))
    assert not bad, "designs outside the same-stream band: %r" % bad[:10]
    return {"designs": len(idx), "hit_difference": tot_diff, "ambiguous_draws": tot_amb, "per_design": rec}


def band(p_exact, n):
    return 5.0 * math.sqrt(max(p_exact * (1.0 - p_exact), 0.0) / n) + 1e-7


def assert_band(p_gpu, p_exact, n, idx):
    """|p_gpu - p_exact| <= 5 SE + 1e-7 per design.  Returns the number of
    designs, the largest and the mean |error| in units of SE, and per design
    p_gpu, p_exact, n and the signed error in SE."""
    bad = [(j, float(p_gpu[j]), float(p_exact[k])) for k, j in enumerate(idx)
           if abs(p_gpu[j] - p_exact[k]) > band(p_exact[k], n if np.isscalar(n) else n[k])]
    assert not bad, "designs outside 5 SE of the exact value: %r" % bad[:10]
    z, rec = [], []
    for k, j in enumerate(idx):
        nn = n if np.isscalar(n) else n[k]
        se = math.sqrt(max(p_exact[k] * (1.0 - p_exact[k]), 1e-300) / nn)
        zk = (float(p_gpu[j]) - float(p_exact[k])) / se
        z.append(abs(zk))
        rec.append({"design": int(j), "p_gpu": float(p_gpu[j]), "p_exact": float(p_exact[k]), "n": int(nn),
                    "z": zk})
    return {"designs": len(idx), "max_abs_z": max(z) if z else 0.0, "mean_abs_z": float(np.mean(z)) if z else 0.0,
            "per_design": rec}
