"""Benchmark of the design-objective engine on one GB300 (or N replicas).

Step = one pass of the whole hot path over the d=3 design grid (16 scenarios
x 64 cutoff quantiles x 64 allocations, 1e6 draws per design, one stream key
per scenario): Cholesky of each Sigma, the fused shared-draw sampling kernel
(Philox -> Box-Muller -> L z once per draw and block, then the indicator and
the likelihood-ratio and sigmoid adjoint sums of every design of the
scenario against it), the FP64 finalisation (p, SE, gradients w.r.t. cutoff,
allocation, delta+, delta-) and the local-quadratic smoothing with argmax.
`per_design_step` times the same step with one stream key per design
(independent draws), where the per-design kernel makes every draw.

Prints one JSON line.  `value` is draw-evaluations per second over the whole
job (all ranks); `roofline` and `pipe_bound` refer to the sampling kernel:
the min-over-pipes bound from its per-draw-evaluation operation counts and
the instruction-class rates this GPU measures (`mcd_pipe_rate`); `e2e`
times the same step through the public API with inputs copied from pinned
host memory and results copied back; `cpu_baseline` times the FP64 oracle
on the host and compares its hit counts with the GPU's at the same seed.
`extras` holds the other configurations (d = 10, 20, the batched uneven
problem, shared draws, FP64 path, smoothing at scale) and the paper's own
workloads (two-layer estimator, FWER calibration, the Sec. 3 sweep).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MC draw-evals/s & % FP32-pipe peak at d=3/10/20; adjoint overhead vs plain"
UNIT = "draw-evals/s"
LANES = 128
SM_MAX_MHZ = 2070.0
WORKLOAD = ("d=3 design grid: 16 scenarios x 64 cutoff quantiles x 64 allocation fractions, "
            "1e6 FP32 draws per design (one stream per scenario), forward + adjoint (cutoff, allocation, "
            "delta+, delta-; sigmoid h=1e-2), FP64 finalisation, local-quadratic smoothing + argmax")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "sample_kernel_c2_traffic.txt")
KERNEL_SOURCES = [os.path.join(ROOT, "paper_2005_10494_gb300", "csrc", f)
                  for f in ("sample.cuh", "rng.cuh", "mcd_internal.cuh")]
SHARED_TRAFFIC_FILE = os.path.join(ROOT, "profiles", "shared_kernel_c2_traffic.txt")
SHARED_SOURCES = [os.path.join(ROOT, "paper_2005_10494_gb300", "csrc", f)
                  for f in ("shared.cuh", "sample.cuh", "rng.cuh", "mcd_internal.cuh")]


# Algorithmic 32-bit operations per draw-evaluation (one design, one draw):
#   Philox4x32-10: 10 rounds x (2 wide multiplies + 2 three-input xors) per 4
#   normals -> 10 per normal; uniform map 2 per normal; Box-Muller 8 per pair
#   (lg2, scale, sqrt, angle fma, sin, cos, 2 products) -> 4 per normal;
#   transform d(d+1)/2 FMA; indicator d compares + 1 count.
#   Adjoint adds 2d + 1 (likelihood-ratio sums) and 7d (sigmoid factors).
def packed_adjoint(d):
    """The FP32 adjoint forms its sigmoid factors and sums two coordinates
    per packed instruction except at d = 16, 18, 20 (csrc/sample.cuh)."""
    return d not in (16, 18, 20)


def adjoint_fp32_ops(d):
    """FP32 instructions of the adjoint per draw: scalar and packed (x2).
    Per coordinate: the sums A and B, the sigmoid argument, 1 + e, 1 - keep
    and the sum G (6), plus the running product (scalar, d).  Packed, the
    four sigmoid terms take floor(d/2) packed and d mod 2 scalar
    instructions each; A and B likewise on the draws whose normals start at
    an even index of their group (all draws at even d, half at odd d), else
    d scalar each."""
    if not packed_adjoint(d):
        return 7.0 * d, 0.0
    half, odd = d // 2, d % 2
    pa = 1.0 if odd == 0 else 0.5
    scalar = 2 * (pa * odd + (1 - pa) * d) + 4 * odd + d
    packed = 2 * pa * half + 4 * half
    return scalar, packed


def ops_per_draw(d, grad):
    ops = 16 * d + d * (d + 1) // 2 + d + 1
    if grad:
        sc, pk = adjoint_fp32_ops(d)
        ops += 2 * d + 1 + sc + pk
    return ops


# FP32 floating-point work per draw-evaluation (FMA = 2): transform d(d+1),
# Box-Muller 5 per pair; adjoint 2 per LR sum pair and 9 per sigmoid factor.
def fp32_flops_per_draw(d, grad):
    f = d * (d + 1) + 5 * d / 2.0
    if grad:
        f += 4 * d + 9 * d
    return f


# Operations per draw-evaluation by instruction class (one design, one draw,
# FP32 path), counted from the estimator as the sampling kernel writes it:
#   Philox4x32-10 per call (4 normals): 19 wide multiplies (round 1's key
#     product is a per-tile constant), 19 xors and 1 counter add (ALU);
#   Box-Muller per pair: 2 word-to-float shift-adds and a compare-select
#     (ALU, 4), 6 FP32 (u0, 2v, log scale, angle, two products), and one
#     each of lg2, sqrt, sin and cos;
#   y = L z: d(d+1)/2 FP32; above d = 6, L comes from shared memory:
#     sum_i ceil((i+1)/4) 16-byte loads per group of G draws (G = 1, 2 or 4
#     draws whose normals fill whole Philox calls; the draws of a group
#     share the loads) and t stays in registers;
#   indicator: d compares and one count add (ALU).
#   Adjoint per coordinate: 7 FP32 (sums A and B; sigmoid argument, 1 + e,
#     running product, 1 - keep, sum G; all but the product two coordinates
#     per packed instruction where packed_adjoint, see adjoint_fp32_ops),
#     ex2, rcp and, above d = 6, one
#     shared load (the scaled threshold); one select per draw (ALU).  At the
#     dimensions where the adjoint reloads with volatile loads, every draw
#     loads all chunks of L and both thresholds.
# An ncu capture of the executed instructions per pipe agrees with these
# counts within 10 % at d = 3, 10 and 20.
def hbm_peak(path=os.path.join(ROOT, "MEASURED_PEAKS.json")):
    """HBM copy bandwidth (GB/s) to judge the smoothing kernel against: the
    measured figure of the GB300s when the file exists, else the
    earlier single measurement of 6.8 TB/s.  Returns (GB/s, source)."""
    try:
        with open(path) as f:
            v = float(json.load(f)["hbm_gbs"])
        if v > 0:
            return v, "measured (MEASURED_PEAKS.json hbm_gbs)"
    except (OSError, ValueError, KeyError, TypeError):
        pass
    return 6800.0, "fallback 6.8 TB/s (no measured figure)"


def class_counts(d, grad):
    calls, pairs = d / 4.0, d / 2.0
    c = {"mul_wide": 19 * calls, "alu": 20 * calls + 4 * pairs + d + 1,
         "ffma": 6 * pairs + d * (d + 1) / 2.0, "ffma2": 0.0, "lg2": pairs, "sqrt": pairs, "sin": pairs,
         "cos": pairs, "ex2": 0.0, "rcp": 0.0, "lds128": 0.0}
    # adjoint kernels that reload the factor (and both thresholds) for
    # every draw: the dimensions of volatile_loads() in sample.cuh
    reload = grad and (8 <= d <= 12 or 15 <= d <= 19)
    if d > 6:
        group = 1 if (d % 4 == 0 or reload) else (2 if d % 2 == 0 else 4)
        c["lds128"] = sum((i + 4) // 4 for i in range(d)) / float(group)
    if grad:
        sc, pk = adjoint_fp32_ops(d)
        c["ffma"] += sc
        c["ffma2"] += pk
        c["ex2"] += d
        c["rcp"] += d
        c["alu"] += 1
        if d > 6:
            c["lds128"] += 2 * d if reload else d
    return c


MUFU = ("lg2", "sqrt", "sin", "cos", "ex2", "rcp")


def shared_class_counts(d, grad, dpt, active=1.0):
    """Operations per draw-evaluation of the shared-draw kernel (csrc/shared.cuh)
    for one design and one draw, by instruction class: the draw itself is
    made once per block for a whole chunk of designs, so its cost vanishes
    per design.  The differences t_i - y_i go two coordinates per packed
    FMA (floor(d/2) `ffma2`, one FP32 subtraction for an odd d); the draw's
    row of y is one 16-byte load per 4 coordinates, shared by the thread's
    dpt designs.  Forward: the or of the d sign words with three-input logic
    (ceil((d-1)/2)) and the count add of the sign bit (ALU).  Adjoint: the
    smallest difference with three-input minima (ceil((d-1)/2)), the hit
    test, the count (select and add; at odd d none, see below), the window
    test |min_i (t_i - y_i)| < w of the sigmoid's reach (one compare of a
    magnitude) and the warp vote (ALU); the sum A over hits (floor(d/2)
    packed adds; at odd d one more, whose second lane counts the hit in the
    z row's padding slot); the row of z; and, in the fraction `active` of
    warp-draws where some lane's draw is within that window, per coordinate
    the exponent, 1 + e, 1 - keep and the FMA of sum G two coordinates per
    packed instruction (4 floor(d/2) `ffma2`, 4 scalar at odd d), the
    running product (d scalar), ex2 and rcp (2d MUFU)."""
    rows = -(-d // 4)
    half, odd = d // 2, d % 2
    c = {"mul_wide": 0.0, "alu": (d - 1 + 1) // 2 + 1.0, "ffma": float(odd), "ffma2": float(half),
         "lg2": 0.0, "sqrt": 0.0, "sin": 0.0, "cos": 0.0, "ex2": 0.0, "rcp": 0.0, "lds128": rows / float(dpt)}
    if grad:
        # at odd d the hit count rides in the last packed add of A (the z
        # row's padding slot holds 1), instead of a select and an add
        c["alu"] = (d - 1 + 1) // 2 + (3.0 if odd else 5.0)
        c["ffma2"] += half + odd
        c["ffma"] += active * (d + 4 * odd)
        c["ffma2"] += active * 4 * half
        c["lds128"] += rows / float(dpt)
        c["ex2"] += active * d
        c["rcp"] += active * d
    return c


def shared_fp32_flops(d, grad, active=1.0):
    """Algorithmic FP32 flops per draw-evaluation of the shared-draw kernel
    (FMA = 2): d differences; the adjoint adds the d sums of A and, where the
    sigmoid is taken, per coordinate its exponent, 1 + e, the product,
    1 - keep and the FMA of G (6d)."""
    f = float(d)
    if grad:
        f += d + 6 * d * active
    return f


def shared_active_fraction(prob, h, draws=1024, warp=32, seed=0):
    """Fraction of (32-design block, draw) pairs of the shared-draw kernel in
    which some design's draw has a sigmoid exponent x_max = max_i (y_i - t_i)
    log2(e) / h with |x_max| < 25.03, i.e. where the kernel evaluates the
    smoothed indicator (elsewhere every contribution is zero or below 3e-8
    and the kernel skips it).  A warp tests 32
    consecutive designs of a group against one draw; estimated on `draws`
    normal draws per scenario (numpy FP64, not the kernel's stream: this is
    a property of the workload)."""
    rng = np.random.default_rng(seed)
    tot = act = 0
    l2e = 1.4426950408889634 / h
    for s in range(prob.n_scen):
        idx = np.flatnonzero(prob.design_scen == s)
        if idx.size == 0:
            continue
        L = np.linalg.cholesky(prob.sigmas[s])
        y = rng.standard_normal((draws, L.shape[0])) @ L.T
        t = np.stack([prob.t(j) for j in idx])
        for w0 in range(0, idx.size, warp):
            xm = ((y[:, None, :] - t[None, w0:w0 + warp, :]) * l2e).max(axis=2)
            a = (np.abs(xm) < 25.03).any(axis=1)
            act += int(a.sum())
            tot += a.size
    return act / max(tot, 1)


def shared_pipe_bound(rates, d, grad, dpt, active, sm_count, mhz=SM_MAX_MHZ):
    """The min-over-pipes bound of the shared-draw kernel (as pipe_bound)."""
    n = shared_class_counts(d, grad, dpt, active)
    r_pk = rates.get("ffma2", rates["ffma"] / 2.0)
    clk = {
        "alu": n["alu"] / rates["lop3"],
        "fp32": n["ffma"] / rates["ffma"] + n["ffma2"] / r_pk,
        "mufu": sum(n[k] / rates[k] for k in MUFU),
        "lsu": n["lds128"] / rates["lds128"],
        "issue": sum(n.values()) / LANES,
    }
    binding = max(clk, key=clk.get)
    return {"sm_clk_per_draw": clk, "binding": binding,
            "bound_draw_evals_per_s": sm_count * mhz * 1e6 / clk[binding], "ops_per_draw": n,
            "active_fraction": active}


def pipe_bound(rates, d, grad, sm_count, mhz=SM_MAX_MHZ):
    """The min-over-pipes bound on draw-evaluations per second: SM clocks per
    draw on each pipe = the draw's operations of that pipe's classes / the
    measured operations per SM clock (mcd_pipe_rate); the busiest pipe binds.
    "fma_pipes" assumes wide multiplies occupy the heavy half of the FMA pipe
    and FP32 work spreads over both halves; "issue" is one warp instruction
    per clock per scheduler (128 operations per SM clock)."""
    n = class_counts(d, grad)
    half = rates["ffma"] / 2.0
    r_pk = rates.get("ffma2", rates["ffma"] / 2.0)
    # wide multiplies: the faster of the bare multiply-add and the multiplies
    # inside Philox rounds as the kernels run them
    r_mul = max(rates["mul_wide"], rates.get("philox", 0.0))
    clk = {
        "int_multiply": n["mul_wide"] / r_mul,
        "alu": n["alu"] / rates["lop3"],
        "fp32": n["ffma"] / rates["ffma"] + n["ffma2"] / r_pk,
        "fma_pipes": (n["mul_wide"] * half / r_mul + n["ffma"]) / rates["ffma"] + n["ffma2"] / r_pk,
        "mufu": sum(n[k] / rates[k] for k in MUFU),
        "lsu": n["lds128"] / rates["lds128"],
        "issue": sum(n.values()) / LANES,
    }
    binding = max(clk, key=clk.get)
    bound = sm_count * mhz * 1e6 / clk[binding]
    return {"sm_clk_per_draw": clk, "binding": binding, "bound_draw_evals_per_s": bound,
            "ops_per_draw": n}


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-extras", action="store_true", help="skip the d=10/20, smoothing and C3 lines")
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="target CPU time of the oracle baseline")
    ap.add_argument("--case", default=None, choices=["c2-small", "c4-small", "c5-small", "smooth", "smooth-f32",
                                                      "c2-shared", "c2-shared-full", "tps", "shared-dims",
                                                      "perdesign-dims", "tps-timing"],
                    help="run a small profiling case (a few launches, no timing), or one of the timing sweeps "
                         "(shared-dims, perdesign-dims, tps-timing: JSON lines), and exit")
    return ap.parse_args()


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        return self.summarise(self.lines)

    @staticmethod
    def summarise(lines):
        """Median SM clock, max SM clock and the throttle reasons seen in
        nvidia-smi CSV lines of FIELDS (malformed lines are skipped)."""
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------ CPU oracle
def host_cpu():
    """Model name and logical core count of the host (lscpu, else /proc/cpuinfo)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        fields = dict(line.split(":", 1) for line in out.splitlines() if ":" in line)
        fields = {k.strip(): v.strip() for k, v in fields.items()}
        model = fields.get("Model name") or fields.get("Vendor ID")
    except (OSError, subprocess.SubprocessError):
        pass
    if not model:
        try:
            with open("/proc/cpuinfo") as f:
                for line in f:
                    if line.lower().startswith(("model name", "cpu part")):
                        model = line.split(":", 1)[1].strip()
                        break
        except OSError:
            pass
    return {"model": model or "unknown", "logical_cores": os.cpu_count()}


def quadrature_times():
    """The deterministic oracle's time per design (FP64, one thread):
    conditioning with nested Gauss-Legendre on the dense d=3 factor (O1) and
    the structured forms -- the one-factor integral (equicorrelated d=3),
    the Markov recursion (AR(1) d=10) and the nested factor integral (block
    d=20) -- on designs of the d=3, d=10 and d=20 grids."""
    import workloads
    from oracle import quad
    cases = []
    for k, (q, a) in enumerate([(0.3, 0.4), (0.6, 0.7), (0.85, 0.25), (0.1, 0.55)]):
        mu, b, _ = workloads.design_at("c2", q, a, scenario=k)
        rho = workloads.c2_scenarios(16)[k][2]
        cases.append(("o1_dense_d3", lambda t=b - mu, r=rho: quad.orthant_dense(t, workloads.equicorrelated(3, r))))
        cases.append(("o2_equi_d3", lambda t=b - mu, r=rho: quad.orthant_equi(t, r)))
    for q, a in [(0.3, 0.4), (0.7, 0.6)]:
        mu, b, _ = workloads.design_at("c4", q, a)
        cases.append(("o2_ar1_d10", lambda t=b - mu: quad.orthant_ar1(t, 0.3)))
        mu, b, _ = workloads.design_at("c5", q, a)
        t5 = workloads.tables()["c5"]
        cases.append(("o2_block_d20", lambda t=b - mu: quad.orthant_block(t, t5["sizes"], t5["rho_in"],
                                                                          t5["rho_out"])))
    acc = {}
    for name, fn in cases:
        t0 = time.perf_counter()
        fn()
        acc.setdefault(name, []).append(time.perf_counter() - t0)
    return {name + "_ms_per_design": 1000.0 * float(np.mean(v)) for name, v in acc.items()}


def cpu_oracle_rate(prob, seconds, h=0.01, seed=0, gpu_hits=None):
    """Time the FP64 oracle (as it stands) on a sample of the workload's designs.
    With gpu_hits (the GPU step's hit counts at the same seed), also report
    the GPU's error against the oracle on those designs: same counters, so
    the counts differ only by draws whose FP32 and FP64 indicators disagree."""
    from oracle import mc as omc
    rng = np.random.default_rng(123)
    idx = rng.choice(prob.n_design, 64, replace=False)
    designs = [{"Sigma": prob.sigmas[prob.design_scen[j]], "t": prob.t(j), "key": int(prob.keys[j]),
                "n_draws": 20_000} for j in idx[:16]]
    t0 = time.perf_counter()
    omc.mc_batch(designs, seed, h=h, grad=True)
    probe = time.perf_counter() - t0
    per_draw = probe / (16 * 20_000)
    n = int(prob.n_draws[0])                                  # full draws per design
    n_des = int(max(16, min(prob.n_design, round(seconds / per_draw / n / 16) * 16)))
    idx = rng.choice(prob.n_design, n_des, replace=False)
    designs = [{"Sigma": prob.sigmas[prob.design_scen[j]], "t": prob.t(j), "key": int(prob.keys[j]),
                "n_draws": n} for j in idx]
    cores = omc.num_threads()
    t0 = time.perf_counter()
    ora = omc.mc_batch(designs, seed, h=h, grad=True)
    dt = time.perf_counter() - t0
    rec = {"value": n_des * n / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
           "sample": "%d random designs of the d=3 grid x %d draws each (their full draw count), "
                     "FP64 estimator with adjoint sums, %.1f s" % (n_des, n, dt)}
    # one thread on a quarter of the time budget: the per-core figure beside
    # the all-core one, and the host it ran on
    n1 = int(max(1, min(n_des, round(seconds / 4.0 / (per_draw * cores) / n))))
    omc.set_num_threads(1)
    try:
        t0 = time.perf_counter()
        omc.mc_batch(designs[:n1], seed, h=h, grad=True)
        dt1 = time.perf_counter() - t0
    finally:
        omc.set_num_threads(cores)
    rec["single_thread"] = {"value": n1 * n / dt1, "unit": UNIT, "cores": 1,
                            "sample": "%d of the designs above, %.1f s" % (n1, dt1)}
    rec["per_core_all_cores"] = rec["value"] / cores
    rec["host"] = host_cpu()
    rec["quadrature"] = quadrature_times()
    if gpu_hits is not None:
        g = np.asarray(gpu_hits, dtype=np.int64)[idx]
        o = np.asarray(ora["hits"], dtype=np.int64)
        diff = np.abs(g - o)
        p = o / float(n)
        se = np.sqrt(np.maximum(p * (1.0 - p), 1e-300) / n)
        rec["gpu_vs_oracle"] = {"designs": int(n_des), "seed": seed, "designs_differing": int(np.count_nonzero(diff)),
                                "max_abs_hit_diff": int(diff.max()), "total_abs_hit_diff": int(diff.sum()),
                                "max_abs_p_diff_over_se": float(np.max(diff / float(n) / se))}
    return rec


# ------------------------------------------------------------ reference
def run_reference(args, rank):
    if rank != 0:
        return
    import workloads
    prob = workloads.c2()
    per_step = max(1.0, min(20.0, 150.0 / max(1, args.steps + args.warmup)))
    from oracle import mc as omc
    rng = np.random.default_rng(7)
    idx = rng.choice(prob.n_design, 32, replace=False)
    probe = [{"Sigma": prob.sigmas[prob.design_scen[j]], "t": prob.t(j), "key": int(prob.keys[j]),
              "n_draws": 10_000} for j in idx[:8]]
    t0 = time.perf_counter()
    omc.mc_batch(probe, 0, h=0.01, grad=True)
    per_draw = (time.perf_counter() - t0) / 80_000
    n = int(max(1000, min(1_000_000, per_step / per_draw / 32)))
    designs = [{"Sigma": prob.sigmas[prob.design_scen[j]], "t": prob.t(j), "key": int(prob.keys[j]),
                "n_draws": n} for j in idx]
    for _ in range(args.warmup):
        omc.mc_batch(designs, 0, h=0.01, grad=True)
    times = []
    for s in range(args.steps):
        t0 = time.perf_counter()
        omc.mc_batch(designs, s + 1, h=0.01, grad=True)
        times.append(time.perf_counter() - t0)
    total = sum(times)
    value = args.steps * 32 * n / total
    sample = "32 designs of the d=3 grid x %d draws per step, FP64 oracle estimator with adjoint sums" % n
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "sample": sample},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": omc.num_threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------ multi-replica runs
def rank_keys(keys, rank):
    """Stream keys of rank `rank`: each replica evaluates its own independent
    copy of the grid (weak scaling; rank 0 keeps the workload's keys)."""
    return np.asarray(keys, dtype=np.uint64) + np.uint64(rank * 1_000_003)


def max_over_ranks(t, device):
    """The slowest rank's time (the only collective besides the barrier)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return t
    x = torch.tensor([t], dtype=torch.float64, device=device)
    dist.all_reduce(x, op=dist.ReduceOp.MAX)
    return float(x.item())


# ------------------------------------------------------------ our arm
def read_record(path, sources):
    """The key: value lines of a committed ncu summary, or None when it is
    missing or the kernel sources no longer hash to its src_sha256."""
    if not os.path.exists(path):
        return None
    rec = {}
    with open(path) as f:
        for ln in f:
            if ":" in ln and not ln.startswith("#"):
                k, v = ln.split(":", 1)
                rec[k.strip()] = v.strip()
    h = hashlib.sha256()
    for p in sources:
        with open(p, "rb") as f:
            h.update(f.read())
    return rec if rec.get("src_sha256") == h.hexdigest() else None


def traffic_record(tiles):
    """DRAM bytes of one per-design sampling launch of `tiles` tiles, from the
    committed ncu capture of a small case (traffic grows with the tile
    count), or None when the kernel sources changed since that capture."""
    rec = read_record(TRAFFIC_FILE, KERNEL_SOURCES)
    if rec is None:
        return None
    try:
        per_tile = (float(rec["dram_bytes_read_small"]) + float(rec["dram_bytes_write_small"])) / float(rec["tiles_small"])
    except (KeyError, ValueError, ZeroDivisionError):
        return None
    return per_tile * tiles


def shared_traffic_record():
    """DRAM bytes of one launch of the shared-draw adjoint kernel on the full
    d=3 grid step, from the committed ncu capture of that launch, or None when
    the kernel sources changed since."""
    rec = read_record(SHARED_TRAFFIC_FILE, SHARED_SOURCES)
    if rec is None:
        return None
    try:
        return float(rec["dram_bytes_read"]) + float(rec["dram_bytes_write"])
    except (KeyError, ValueError):
        return None


def kernel_rate(pkg, ctx, prob, grad, reps=2, h=0.01):
    """Draw-evals/s of the sampling kernel alone on one workload (CUDA events)."""
    import torch
    dp = pkg.DeviceProblem.from_workload(prob)
    plan = pkg.Plan(ctx, dp, grad=grad, k=4 if grad else 0, timing=True, autotune=True)
    jac = torch.as_tensor(prob.jac_packed(), dtype=torch.float64, device="cuda") if grad else None
    best = 1e30
    for r in range(reps + 1):
        if grad:
            plan.grad(100 + r, jac, h)
        else:
            plan.eval(100 + r)
        ms = plan.kernel_ms()
        if r > 0:
            best = min(best, ms)
    ctx.sync_status()
    plan.close()
    return prob.total_draws() / (best / 1e3), best


def shared_dpt(d, grad):
    """Designs per thread of the shared-draw kernel (SharedShape in shared.cuh)."""
    if grad:
        return 4 if d <= 4 else (2 if d <= 8 else 1)
    return 4 if d <= 10 else 2


def timed_steps(step, steps, stream, flush, kernel_ms):
    """Run `steps` steps bracketed by CUDA events on `stream`, flushing L2
    before each; returns (per-step ms, per-step sampling-kernel ms, wall s)."""
    import torch
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    kms = []
    wall0 = time.perf_counter()
    for s in range(steps):
        flush.fill_(float(s))                 # evict L2 between steps (256 MB > 126 MB L2)
        ev[s][0].record(stream)
        step(s)
        ev[s][1].record(stream)
        kms.append(kernel_ms())               # waits for this step
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in ev], kms, time.perf_counter() - wall0


def per_design_step(pkg, ctx, args, rates, sm_count, stream, flush):
    """The same step with independent stream keys (one per design): the
    per-design kernel (Philox -> Box-Muller -> L z -> indicator -> sums per
    draw and design), timed like the headline step, with its roofline."""
    import torch

    import workloads
    prob = workloads.c2(keys="independent")
    dp = pkg.DeviceProblem.from_workload(prob)
    jac = torch.as_tensor(prob.jac_packed(), dtype=torch.float64, device="cuda")
    plan = pkg.Plan(ctx, dp, grad=True, k=4, autotune=True, graph=True, timing=True)
    S, G1, G2 = prob.n_scen, prob.grid[0], prob.grid[1]

    def step(seed):
        out = plan.grad(seed, jac, 0.01, stream=stream)
        pkg.mc_smooth_argmax(ctx, out["p"], S, G1, G2, bandwidth=3.0, degree=2, stream=stream)

    for w in range(args.warmup):
        step(2000 + w)
    torch.cuda.synchronize()
    step_ms, kms, _ = timed_steps(step, args.steps, stream, flush, plan.kernel_ms)
    ctx.sync_status()
    draws = prob.total_draws()
    kernel_ms = statistics.mean(kms)
    ops = ops_per_draw(3, True)
    peak_ops = sm_count * LANES * SM_MAX_MHZ * 1e6
    achieved = ops * draws / (kernel_ms / 1e3)
    pb = pipe_bound(rates, 3, True, sm_count)
    rate = draws / (kernel_ms / 1e3)
    fp32 = fp32_flops_per_draw(3, True) * rate
    fp32_peak = sm_count * LANES * 2 * SM_MAX_MHZ * 1e6
    cfg3 = plan.config(3)
    res = {"workload": "the headline step with one stream key per design (independent draws): "
                       "per-design sampling kernel",
           "value": args.steps * draws / (sum(step_ms) / 1e3), "unit": UNIT, "ms_per_step": statistics.mean(step_ms),
           "launch": {"threads": cfg3["threads"], "tile_draws": cfg3["tile_draws"],
                      "blocks_per_sm": cfg3["blocks_per_sm"], "tiles": plan.tiles()},
           "roofline": {"bound": "issue", "achieved": achieved / 1e9, "peak": peak_ops / 1e9, "unit": "Gop/s",
                        "frac": achieved / peak_ops, "traffic": traffic_record(plan.tiles()),
                        "kernel": "sample_kernel_4b<3,3,grad,float>", "kernel_ms": kernel_ms, "ops_per_draw": ops,
                        "peak_basis": "%d SMs x 128 issue slots x %.0f MHz (max SM clock): one warp "
                                      "instruction per scheduler per clock" % (sm_count, SM_MAX_MHZ)},
           "pipe_bound": {"kernel": "sample_kernel_4b<3,3,grad,float>", "achieved": rate,
                          "bound": pb["bound_draw_evals_per_s"], "unit": UNIT,
                          "frac": rate / pb["bound_draw_evals_per_s"], "binding": pb["binding"],
                          "sm_clk_per_draw": pb["sm_clk_per_draw"], "ops_per_draw": pb["ops_per_draw"]},
           "fp32_pipe": {"achieved_tflops": fp32 / 1e12, "peak_tflops": fp32_peak / 1e12, "frac": fp32 / fp32_peak,
                         "flops_per_draw": fp32_flops_per_draw(3, True)}}
    plan.close()
    return res


def run_ours(args, rank, world):
    import torch

    import paper_2005_10494_gb300 as pkg
    import workloads

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    ctx = pkg.Context(dev.index)
    # the d=3 grid with one stream key per scenario: the 4096 designs of a
    # scenario share their draws (common random numbers), so the plan takes
    # the shared-draw kernel; hit counts are those of the per-design kernel
    prob = workloads.c2()
    if world > 1:
        prob.keys = rank_keys(prob.keys, rank)
    dp = pkg.DeviceProblem.from_workload(prob)
    jac = torch.as_tensor(prob.jac_packed(), dtype=torch.float64, device=dev)
    plan = pkg.Plan(ctx, dp, grad=True, k=4, graph=True, timing=True, shared=True)
    S, G1, G2 = prob.n_scen, prob.grid[0], prob.grid[1]
    stream = torch.cuda.Stream(device=dev)      # capturable stream for the plan's CUDA graph
    stream.wait_stream(torch.cuda.current_stream())
    torch.cuda.set_stream(stream)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def step(seed):
        out = plan.grad(seed, jac, 0.01, stream=stream)
        sm = pkg.mc_smooth_argmax(ctx, out["p"], S, G1, G2, bandwidth=3.0, degree=2, stream=stream)
        return out, sm

    for w in range(args.warmup):
        step(1000 + w)
    ctx.sync_status()
    torch.cuda.synchronize()

    clocks = ClockSampler(dev.index)
    if rank == 0:
        clocks.start()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    step_ms, kms, wall = timed_steps(step, args.steps, stream, flush, plan.kernel_ms)
    t_total = sum(step_ms) / 1e3
    t_total = max_over_ranks(t_total, dev)
    clk = clocks.stop() if rank == 0 else None
    ctx.sync_status()

    draws = prob.total_draws()
    value = world * args.steps * draws / t_total
    kernel_ms = statistics.mean(kms)
    if rank != 0:
        return

    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    rate = draws / (kernel_ms / 1e3)
    # instruction-class rates of this GPU (own microbenchmarks), for the
    # min-over-pipes bounds
    rates = pkg.pipe_rates(ctx, iters=4096, stream=stream)
    active = shared_active_fraction(prob, 0.01, draws=512)
    dpt = shared_dpt(3, True)
    spb = shared_pipe_bound(rates, 3, True, dpt, active, sm_count)
    n = spb["ops_per_draw"]
    fp32_flops = shared_fp32_flops(3, True, active)
    fp32 = fp32_flops * rate
    fp32_peak = sm_count * LANES * 2 * SM_MAX_MHZ * 1e6

    # e2e: same step through the public API from pinned host buffers
    f64 = torch.float64
    h_sig = torch.as_tensor(prob.sigma_packed(), dtype=f64).pin_memory()
    h_mu = torch.as_tensor(prob.mu_packed(), dtype=f64).pin_memory()
    h_b = torch.as_tensor(prob.b_packed(), dtype=f64).pin_memory()
    h_jac = torch.as_tensor(prob.jac_packed(), dtype=f64).pin_memory()
    J = prob.n_design
    outs_h = {"p": torch.empty(J, dtype=f64).pin_memory(), "hits": torch.empty(J, dtype=torch.int64).pin_memory(),
              "grad_lr": torch.empty(4 * J, dtype=f64).pin_memory(), "grad_sig": torch.empty(4 * J, dtype=f64).pin_memory(),
              "grad_se": torch.empty(4 * J, dtype=f64).pin_memory(), "smoothed": torch.empty(J, dtype=f64).pin_memory(),
              "argmax_idx": torch.empty(S, dtype=torch.int64).pin_memory(),
              "argmax_val": torch.empty(S, dtype=f64).pin_memory()}
    h2d = sum(t.numel() * t.element_size() for t in (h_sig, h_mu, h_b, h_jac))
    d2h = sum(t.numel() * t.element_size() for t in outs_h.values())
    torch.cuda.synchronize()
    e2e_times = []
    for s in range(args.steps):
        flush.fill_(float(s))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        dp.Sigma.copy_(h_sig, non_blocking=True)
        dp.mu.copy_(h_mu, non_blocking=True)
        dp.b.copy_(h_b, non_blocking=True)
        jac.copy_(h_jac, non_blocking=True)
        out, sm = step(500 + s)
        for name in ("p", "hits", "grad_lr", "grad_sig", "grad_se"):
            outs_h[name].copy_(out[name], non_blocking=True)
        for name in ("smoothed", "argmax_idx", "argmax_val"):
            outs_h[name].copy_(sm[name], non_blocking=True)
        torch.cuda.synchronize()
        e2e_times.append(time.perf_counter() - t0)
    e2e_value = world * draws * args.steps / sum(e2e_times)

    out0, _ = step(0)                       # the first timed step's seed, for the oracle comparison
    hits0 = out0["hits"].cpu().numpy()
    ctx.sync_status()

    per = per_design_step(pkg, ctx, args, rates, sm_count, stream, flush)
    # the per-design kernel on the same (common-random-number) keys gives
    # the same hit counts
    ref_plan = pkg.Plan(ctx, dp, graph=False)
    same_hits = bool(np.array_equal(ref_plan.eval(0, stream=stream)["hits"].cpu().numpy(), hits0))
    ref_plan.close()
    ctx.sync_status()

    extras = {}
    if not args.no_extras:
        extras = run_extras(pkg, ctx, prob, rates, sm_count)

    cpu = cpu_oracle_rate(prob, args.cpu_seconds, gpu_hits=hits0)

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * t_total / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "designs": int(J), "draws_per_design": int(prob.n_draws[0]),
                   "d": 3, "parallelism": "replicas" if world > 1 else "single-gpu",
                   "stream_keys": "one per scenario (common random numbers): shared-draw kernel",
                   "l2": "flushed between steps (256 MB write); inputs and outputs are < 20 MB",
                   "launch": {"kernel": "shared_kernel<3,grad>", "designs_per_thread": dpt, "cuda_graph": True}},
        "roofline": {"bound": spb["binding"], "achieved": rate, "peak": spb["bound_draw_evals_per_s"],
                     "unit": UNIT, "frac": rate / spb["bound_draw_evals_per_s"],
                     "traffic": shared_traffic_record(), "kernel": "shared_kernel<3,grad>", "kernel_ms": kernel_ms,
                     "peak_basis": "min over pipes (issue 128 per SM clock; ALU, FP32, MUFU and shared-load "
                                   "rates measured by mcd_pipe_rate) of the per-draw-evaluation operation counts, "
                                   "%d SMs x %.0f MHz; the sigmoid's exponentials in the measured fraction "
                                   "%.3f of warp-draws that reach it" % (sm_count, SM_MAX_MHZ, active)},
        "pipe_bound": {"kernel": "shared_kernel<3,grad>", "achieved": rate, "bound": spb["bound_draw_evals_per_s"],
                       "unit": UNIT, "frac": rate / spb["bound_draw_evals_per_s"], "binding": spb["binding"],
                       "sm_clk_per_draw": spb["sm_clk_per_draw"], "ops_per_draw": n,
                       "active_fraction": active, "rates_ops_per_sm_clk": rates},
        "fp32_pipe": {"achieved_tflops": fp32 / 1e12, "peak_tflops": fp32_peak / 1e12, "frac": fp32 / fp32_peak,
                      "flops_per_draw": fp32_flops},
        "hits_equal_per_design_kernel": same_hits,
        "per_design_step": per,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        # per step: Cholesky, sampling, finalisation, smoothing weights,
        # stencil and argmax
        "gpu_launches": args.steps * 6,
        "clocks": clk,
        "wall_s_timed": wall,
        "cpu_baseline": cpu,
        "extras": extras,
    }
    print(json.dumps(line), flush=True)


def c3_batched_vs_per_design(pkg, ctx, n_sub=512):
    """C3 (256 scenarios, d = 3..10, 38k designs): the whole batch in one
    persistent graph-replayed launch, and on an evenly spaced subsample the
    same designs as one launch each; hits must agree exactly."""
    import torch

    import workloads
    prob = workloads.c3()
    stream = torch.cuda.current_stream()
    dp = pkg.DeviceProblem.from_workload(prob)
    plan = pkg.Plan(ctx, dp, autotune=True, graph=True)
    plan.eval(1, stream=stream)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    full = plan.eval(2, stream=stream)
    b.record(stream)
    b.synchronize()
    full_ms = a.elapsed_time(b)
    full_hits = full["hits"].cpu().numpy()
    plan.close()
    idx = np.linspace(0, prob.n_design - 1, n_sub).astype(int)
    sub = prob.subset(idx)
    sdp = pkg.DeviceProblem.from_workload(sub)
    batched = pkg.Plan(ctx, sdp, graph=True)
    batched.eval(2, stream=stream)
    singles = []
    for j in range(n_sub):
        one = prob.subset([int(idx[j])])
        odp = pkg.DeviceProblem.from_workload(one)
        singles.append((pkg.Plan(ctx, odp), odp))
    torch.cuda.synchronize()
    a.record(stream)
    sb = batched.eval(2, stream=stream)
    b.record(stream)
    b.synchronize()
    batched_ms = a.elapsed_time(b)
    outs = []
    a.record(stream)
    for pl, _ in singles:
        outs.append(pl.eval(2, stream=stream, out={"hits": torch.empty(1, dtype=torch.int64, device="cuda"),
                                                  "p": torch.empty(1, dtype=torch.float64, device="cuda"),
                                                  "se": torch.empty(1, dtype=torch.float64, device="cuda")}))
    b.record(stream)
    b.synchronize()
    single_ms = a.elapsed_time(b)
    ctx.sync_status()
    single_hits = np.array([int(o["hits"].item()) for o in outs])
    equal = bool(np.array_equal(single_hits, sb["hits"].cpu().numpy())
                 and np.array_equal(single_hits, full_hits[idx]))
    for pl, _ in singles:
        pl.close()
    batched.close()
    draws_sub = float(sub.n_draws.astype(np.float64).sum())
    return {"designs": int(prob.n_design), "draws": float(prob.total_draws()), "batched_ms": full_ms,
            "batched_draw_evals_per_s": prob.total_draws() / (full_ms / 1e3),
            "subsample": {"designs": n_sub, "draws": draws_sub, "one_launch_ms": batched_ms,
                          "per_design_launches_ms": single_ms, "speedup": single_ms / batched_ms,
                          "hits_bit_identical": equal}}


def c4_search(pkg, ctx):
    """Gradient-driven search on the d=10 grid's design space (projected Adam,
    likelihood-ratio adjoint, common random numbers)."""
    import torch

    import workloads
    from paper_2005_10494_gb300 import search
    prob = workloads.c4(g1=2, g2=2, n_draws=10)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    x, p_hat, hist = search.gradient_search(ctx, lambda v: workloads.design_at("c4", v[0], v[1]), prob.sigmas[0],
                                            x0=(0.5, 0.5), lo=(0.05, 0.2), hi=(0.95, 0.8), n_draws=10_000_000,
                                            steps=120)
    dt = time.perf_counter() - t0
    return {"steps": 120, "draws_per_step": 10_000_000, "seconds": dt, "q": float(x[0]), "a": float(x[1]),
            "p_hat": p_hat}


def paper_problem(pkg, ctx, n_alpha=2000, N1=10240, N2=20480):
    """One optimisation problem of the paper at its own sizes (Sec. 2.2-3):
    n_alpha alpha points, each estimated by the two-layer estimator with N1
    prior samples crossed with N2 inner draws (strong-biomarker condition,
    d = 3); all outer samples share the inner draws, so the shared-draw
    kernel evaluates N1 * N2 pairs per alpha point from N2 draws."""
    import torch

    import workloads
    a = workloads.paper_two_layer_arrays("c", N1=N1, N2=N2, alphas=workloads.paper_alpha_points("c", n_alpha), seed=0)
    J, d = a["mu"].shape
    f64 = torch.float64
    t0 = time.perf_counter()
    dp = pkg.DeviceProblem(np.array([d], np.int32), np.zeros(J, np.int32), np.full(J, N2, np.uint64),
                           np.zeros(J, np.uint64), torch.as_tensor(a["sigma"].ravel(), dtype=f64, device="cuda"),
                           torch.as_tensor(a["mu"].ravel(), dtype=f64, device="cuda"),
                           torch.as_tensor(a["b"].ravel(), dtype=f64, device="cuda"))
    plan = pkg.Plan(ctx, dp, shared=True)
    plan_s = time.perf_counter() - t0
    plan.eval(1)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ev[0].record()
    out = plan.eval(2)
    ev[1].record()
    ev[1].synchronize()
    ms = ev[0].elapsed_time(ev[1])
    ctx.sync_status()
    p_first = float(out["p"][:N1].mean().item())
    plan.close()
    del dp, out
    # the same alpha point by the per-design kernel (every design draws its own copy of the stream)
    one = workloads.paper_two_layer("c", N1=N1, N2=N2, seed=0, key=0)
    odp = pkg.DeviceProblem.from_workload(one)
    per = pkg.Plan(ctx, odp)
    per.eval(1)
    ev[0].record()
    per.eval(2)
    ev[1].record()
    ev[1].synchronize()
    per_ms = ev[0].elapsed_time(ev[1])
    per.close()
    torch.cuda.empty_cache()
    pairs = float(J) * N2
    return {"alpha_points": n_alpha, "N1": N1, "N2": N2, "pairs": pairs, "ms": ms,
            "pair_evals_per_s": pairs / (ms / 1e3), "plan_build_s": plan_s,
            "per_design_kernel_ms_per_alpha_point": per_ms,
            "per_design_kernel_ms_per_problem_extrapolated": per_ms * n_alpha,
            "p_hat_first_alpha_point": p_first,
            "paper_context": "mean 31.6 s per problem for the whole optimisation on a V100 (Sec. 3; 4.5 h / 513 problems)"}


def shared_line(pkg, ctx, prob, d, rates, sm_count, h=0.01):
    """A grid whose designs share one stream per scenario (common random
    numbers) evaluated by the shared-draw kernel, forward and forward +
    adjoint, against the per-design kernel on the same seed (hits must
    agree); each with its min-over-pipes bound and FP32-pipe fraction."""
    import torch
    dp = pkg.DeviceProblem.from_workload(prob)
    jac = torch.as_tensor(prob.jac_packed(), dtype=torch.float64, device="cuda")
    res = {}
    ref = pkg.Plan(ctx, dp)
    ref_hits = ref.eval(77)["hits"].clone()
    ref.close()
    active = shared_active_fraction(prob, h, draws=256)
    fp32_peak = sm_count * LANES * 2 * SM_MAX_MHZ * 1e6
    for grad in (False, True):
        plan = pkg.Plan(ctx, dp, shared=True, grad=grad, k=4 if grad else 0, timing=True)
        run = (lambda s: plan.grad(s, jac, h)) if grad else (lambda s: plan.eval(s))
        run(76)
        out = run(77)
        ms = plan.kernel_ms()
        same = bool(torch.equal(out["hits"], ref_hits))
        rate = prob.total_draws() / (ms / 1e3)
        pb = shared_pipe_bound(rates, d, grad, shared_dpt(d, grad), active, sm_count)
        res["adj" if grad else "fwd"] = {"kernel_ms": ms, "draw_evals_per_s": rate,
                                         "hits_equal_per_design_kernel": same,
                                         "pipe_bound": {"binding": pb["binding"], "bound": pb["bound_draw_evals_per_s"],
                                                        "frac": rate / pb["bound_draw_evals_per_s"]},
                                         "fp32_pipe_frac": rate * shared_fp32_flops(d, grad, active) / fp32_peak}
        plan.close()
    res["adjoint_overhead"] = res["fwd"]["draw_evals_per_s"] / res["adj"]["draw_evals_per_s"]
    res["active_fraction"] = active
    ctx.sync_status()
    return res


def c5_fp64(pkg, ctx):
    """C5 (d=20) on its 64-design subsample at 1e7 draws per design: the
    all-FP64 sampling path against the FP32 path on the same streams."""
    import workloads
    c5 = workloads.c5()
    sub = c5.subset(workloads.c5_subsample().tolist())
    res, hits = {}, {}
    for name, fp64 in (("fp32", False), ("fp64", True)):
        dp = pkg.DeviceProblem.from_workload(sub)
        plan = pkg.Plan(ctx, dp, fp64=fp64, timing=True)
        best = 1e30
        for r in range(3):
            out = plan.eval(200)
            ms = plan.kernel_ms()
            if r > 0:
                best = min(best, ms)
        hits[name] = out["hits"].cpu().numpy().astype(np.int64)
        res[name] = {"ms": best, "draw_evals_per_s": sub.total_draws() / (best / 1e3)}
        plan.close()
    ctx.sync_status()
    diff = np.abs(hits["fp32"] - hits["fp64"])
    res["fp64_over_fp32_time"] = res["fp64"]["ms"] / res["fp32"]["ms"]
    res["same_stream_hits"] = {"designs": int(diff.size), "designs_differing": int(np.count_nonzero(diff)),
                               "max_abs_diff": int(diff.max()), "total_abs_diff": int(diff.sum()),
                               "draws_per_design": int(sub.n_draws[0])}
    return res


def fwer_calibration(pkg, ctx, n=10_000_000, rounds=14):
    """Eq. 2 on the device: the alpha scale of every split of the d=3 grid's
    16 scenarios x 129 allocations, 1e7 draws per evaluation, against the
    oracle's quadrature calibration (stored tables)."""
    import torch

    import workloads
    prob, w, ref, _ = workloads.fwer_calibration("c2", n_draws=n)
    dp = pkg.DeviceProblem.from_workload(prob)
    wt = torch.as_tensor(w, dtype=torch.float64, device="cuda")
    pkg.mc_fwer_calibrate(ctx, dp, wt, workloads.ALPHA0, rounds=rounds, seed=1)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ev[0].record()
    out = pkg.mc_fwer_calibrate(ctx, dp, wt, workloads.ALPHA0, rounds=rounds, seed=2)
    ev[1].record()
    ev[1].synchronize()
    ctx.sync_status()
    sc = out["scale"].cpu().numpy()
    fw = out["fwer"].cpu().numpy()
    return {"designs": int(prob.n_design), "draws_per_eval": n, "rounds": rounds, "ms": ev[0].elapsed_time(ev[1]),
            "max_rel_err_scale": float(np.max(np.abs(sc - ref) / ref)),
            "rms_rel_err_scale": float(np.sqrt(np.mean(((sc - ref) / ref) ** 2))),
            "max_abs_fwer_minus_alpha0": float(np.max(np.abs(fw - workloads.ALPHA0))),
            "fwer_se_per_eval": float(np.sqrt(workloads.ALPHA0 * (1 - workloads.ALPHA0) / n))}


def paper_optimisation(pkg, ctx):
    """The paper's design optimisation (Sec. 2.1-2.4, 3): alpha at the
    strong condition's reported populations r = (1, 0.446, 0.168) from 2000
    splits (FWER calibration on the device, expected power from shared
    draws, thin-plate spline, its maximiser); then the choice of r over the
    paper's 171 pairs (r2 > r3 on a 0.05 grid) and a spline of the optimal
    power over them, for each of the three conditions of the Sec. 3 sweep."""
    import torch
    from paper_2005_10494_gb300 import search
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    one = search.optimise_alpha(ctx, "c", (1.0, 0.446, 0.168), n3=2000, n_draws=10_000_000, seed=0)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    full = search.optimise_design(ctx, "c", n3=2000, n_draws=4_000_000, seed=0)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    # the rest of the Sec. 3 sweep: conditions (a) and (b), 171 pairs each
    others = {}
    for cond in ("a", "b"):
        ta = time.perf_counter()
        o = search.optimise_design(ctx, cond, n3=2000, n_draws=4_000_000, seed=0)
        torch.cuda.synchronize()
        others[cond] = {"seconds": time.perf_counter() - ta, "r": list(o["r"]),
                        "alpha": [float(a) for a in o["alpha"]], "p_fit": o["p_fit"]}
    sweep = (t2 - t1) + sum(v["seconds"] for v in others.values())
    return {"alpha_at_paper_r": {"seconds": t1 - t0, "alpha": [float(a) for a in one["alpha"]],
                                 "p_fit": one["p_fit"], "paper_alpha": [0.00194, 0.0135, 0.0133],
                                 "paper_power": 0.977},
            "choice_of_r_171_pairs": {"seconds": t2 - t1, "r": list(full["r"]),
                                      "alpha": [float(a) for a in full["alpha"]], "p_fit": full["p_fit"],
                                      "paper_r": [1.0, 0.446, 0.168],
                                      "paper_context": "Sec. 3: about 31.6 s per alpha optimisation on a V100, "
                                                       "171 of them per condition"},
            "other_conditions": others,
            "sweep_513_problems": {"seconds": sweep, "problems": 513,
                                   "note": "171 pairs per condition, plus one alpha optimisation at each chosen r",
                                   "paper_context": "Sec. 3: 4.5 h for the 513 problems on a V100 (context only)"}}


def dim_line(rf, rg, d, rates, sm_count):
    bf, bg = pipe_bound(rates, d, False, sm_count), pipe_bound(rates, d, True, sm_count)
    fp32_peak = sm_count * LANES * 2 * SM_MAX_MHZ * 1e6
    return {"fwd": rf, "adj": rg, "adjoint_overhead": rf / rg,
            "fwd_op_frac": rf * ops_per_draw(d, False) / (sm_count * LANES * SM_MAX_MHZ * 1e6),
            "adj_op_frac": rg * ops_per_draw(d, True) / (sm_count * LANES * SM_MAX_MHZ * 1e6),
            "fwd_fp32_pipe_frac": rf * fp32_flops_per_draw(d, False) / fp32_peak,
            "adj_fp32_pipe_frac": rg * fp32_flops_per_draw(d, True) / fp32_peak,
            "fwd_pipe_bound": {"binding": bf["binding"], "bound": bf["bound_draw_evals_per_s"],
                               "frac": rf / bf["bound_draw_evals_per_s"]},
            "adj_pipe_bound": {"binding": bg["binding"], "bound": bg["bound_draw_evals_per_s"],
                               "frac": rg / bg["bound_draw_evals_per_s"]}}


def run_extras(pkg, ctx, c2, rates, sm_count):
    import torch

    import workloads
    ex = {}
    r3f, _ = kernel_rate(pkg, ctx, c2, grad=False)
    r3g, _ = kernel_rate(pkg, ctx, c2, grad=True)
    ex["d3"] = dim_line(r3f, r3g, 3, rates, sm_count)
    c4 = workloads.c4()
    r10f, _ = kernel_rate(pkg, ctx, c4, grad=False, reps=1)
    r10g, _ = kernel_rate(pkg, ctx, c4, grad=True, reps=1)
    ex["d10"] = dim_line(r10f, r10g, 10, rates, sm_count)
    c5 = workloads.c5()
    r20f, _ = kernel_rate(pkg, ctx, c5, grad=False, reps=1)
    r20g, _ = kernel_rate(pkg, ctx, c5, grad=True, reps=1)
    ex["d20"] = dim_line(r20f, r20g, 20, rates, sm_count)
    # the all-FP64 sampling path (C5 subsample) against the FP32 path
    ex["c5_fp64"] = c5_fp64(pkg, ctx)
    # batched uneven dimensions: one persistent launch vs one launch per design
    ex["c3"] = c3_batched_vs_per_design(pkg, ctx)
    # d=10 gradient search (120 adjoint launches of 1e7 draws)
    ex["c4_search"] = c4_search(pkg, ctx)
    # the grids with one stream per scenario by the shared-draw kernel:
    # d=3 (the step's grid), d=10 (AR(1), 1024 designs x 1e7) and d=20
    # (block, 4096 designs x 1e7)
    ex["c2_shared"] = shared_line(pkg, ctx, c2, 3, rates, sm_count)
    ex["c4_shared"] = shared_line(pkg, ctx, c4, 10, rates, sm_count)
    ex["c5_shared"] = shared_line(pkg, ctx, c5, 20, rates, sm_count)
    # one of the paper's optimisation problems at its own sizes (two-layer estimator)
    ex["paper_problem"] = paper_problem(pkg, ctx)
    # FWER constraint (Eq. 2) solved on the device for every split of the d=3 grid
    ex["fwer_calibration"] = fwer_calibration(pkg, ctx)
    # the paper's whole design optimisation (alpha, then the nested populations)
    ex["paper_optimisation"] = paper_optimisation(pkg, ctx)
    # smoothing at scale: 4096 scenarios x 256 x 256 FP64 grids
    S, G = 4096, 256
    v = torch.rand(S * G * G, dtype=torch.float64, device="cuda")
    best = 1e30
    for r in range(4):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        pkg.mc_smooth_argmax(ctx, v, S, G, G, bandwidth=3.0, degree=2)
        b.record()
        b.synchronize()
        if r > 0:
            best = min(best, a.elapsed_time(b))
    ctx.sync_status()
    nbytes = 16.0 * S * G * G
    peak, source = hbm_peak()
    ex["smoothing"] = {"grid": "4096 x 256 x 256 FP64", "ms": best, "GBps": nbytes / (best / 1e3) / 1e9,
                       "bytes_algorithmic": nbytes, "frac_of_hbm": nbytes / (best / 1e3) / 1e9 / peak,
                       "hbm_peak_GBps": peak, "hbm_peak_source": source}
    # the same grids as FP32 values in and out (mc_smooth_argmax_f32)
    v32 = v.float()
    del v
    best32 = 1e30
    for r in range(4):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        pkg.mc_smooth_argmax(ctx, v32, S, G, G, bandwidth=3.0, degree=2)
        b.record()
        b.synchronize()
        if r > 0:
            best32 = min(best32, a.elapsed_time(b))
    ctx.sync_status()
    nb32 = 8.0 * S * G * G
    ex["smoothing_f32"] = {"grid": "4096 x 256 x 256 FP32", "ms": best32, "GBps": nb32 / (best32 / 1e3) / 1e9,
                           "bytes_algorithmic": nb32, "frac_of_hbm": nb32 / (best32 / 1e3) / 1e9 / peak,
                           "grid_points_per_s": S * G * G / (best32 / 1e3),
                           "speedup_over_fp64": best / best32, "hbm_peak_GBps": peak}
    del v32
    torch.cuda.empty_cache()
    return ex


def _best_kernel_ms(make_plan, run, reps=3):
    """Best of `reps` plan launches, the plan's own CUDA-event kernel time."""
    import torch
    best, out = float("inf"), None
    for _ in range(reps):
        plan = make_plan()
        out = run(plan)
        torch.cuda.synchronize()
        best = min(best, plan.kernel_ms())
        plan.close()
    return best, out


def run_timing_case(case, pkg, ctx):
    """Timing sweeps behind the per-dimension layout choices and the spline
    timings: one JSON line per configuration (CUDA events, best of three)."""
    import torch

    import workloads
    if case == "shared-dims":
        # shared-draw kernel: one LKJ(2) scenario per d with 2048 designs on
        # one stream (common random numbers), 2e6 draws, h = 1e-2
        for d in range(1, 21):
            prob = workloads.crn_groups(np.random.default_rng(d), d_list=[d], group=2048, extra=0,
                                        n_draws=2_000_000, draw_begin=0)
            dp = pkg.DeviceProblem.from_workload(prob)
            line = {"case": case, "d": d, "designs": prob.n_design, "draws": 2_000_000}
            for grad in (False, True):
                ms, out = _best_kernel_ms(lambda: pkg.Plan(ctx, dp, grad=grad, timing=True, shared=True),
                                          lambda plan: plan.grad(3, None, 0.01) if grad else plan.eval(3))
                line["adj" if grad else "fwd"] = prob.total_draws() / (ms * 1e-3)
            print(json.dumps(line), flush=True)
        return
    if case == "perdesign-dims":
        # per-design kernel: 64 designs of one AR(1) scenario (rho 0.3) with
        # their own stream keys, 4e6 draws each
        for d in range(1, 21):
            rng = np.random.default_rng(d)
            J, N = 64, 4_000_000
            prob = workloads.Problem("dims", [workloads.ar1(d, 0.3)], [0] * J,
                                     [rng.normal(0.3, 0.3, d) for _ in range(J)], [np.full(d, 2.2) for _ in range(J)],
                                     [N] * J, np.arange(J) + 5)
            dp = pkg.DeviceProblem.from_workload(prob)
            line = {"case": case, "d": d, "designs": J, "draws": N}
            for grad in (False, True):
                ms, out = _best_kernel_ms(lambda: pkg.Plan(ctx, dp, grad=grad, timing=True),
                                          lambda plan: plan.grad(1, None, 0.01) if grad else plan.eval(1))
                line["adj" if grad else "fwd"] = J * N / (ms * 1e-3)
            print(json.dumps(line), flush=True)
        return
    # tps-timing: the spline fit and its maximiser at the paper's 2000 points
    # (k = 2, 3) and at 4096 (k = 2), smoothing 0.01 (fit) and 1e-6 (maximiser)
    for N, k in ((2000, 2), (2000, 3), (4096, 2)):
        rng = np.random.default_rng(N + k)
        xs = rng.uniform(0, 1, (1, N, k))
        x = torch.as_tensor(xs, dtype=torch.float64, device="cuda")
        y = torch.as_tensor(np.exp(-3.0 * ((xs[0] - 0.55) ** 2).sum(1))[None] + rng.normal(0, 0.01, (1, N)),
                            dtype=torch.float64, device="cuda")
        lo = torch.zeros(k, dtype=torch.float64, device="cuda")
        hi = torch.ones(k, dtype=torch.float64, device="cuda")
        t_fit, t_max = [], []
        for rep in range(4):
            a, b, c = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            a.record()
            pkg.mc_tps_fit(ctx, x, y, smoothing=0.01)
            b.record()
            fit = pkg.mc_tps_fit(ctx, x, y, smoothing=1e-6)
            torch.cuda.synchronize()
            c0 = torch.cuda.Event(enable_timing=True)
            c0.record()
            am = pkg.mc_tps_argmax(ctx, x, fit, lo, hi, iters=300)
            c.record()
            c.synchronize()
            if rep > 0:
                t_fit.append(a.elapsed_time(b))
                t_max.append(c0.elapsed_time(c))
        ctx.sync_status()
        print(json.dumps({"case": case, "points": N, "k": k, "fit_ms": min(t_fit), "argmax_ms": min(t_max),
                          "argmax_x": am["x"].cpu().numpy().ravel().tolist(), "argmax_f": float(am["f"].item())}),
              flush=True)


def run_case(case):
    """Small cases for profilers: a few launches of one kernel, inputs > L2."""
    import torch

    import paper_2005_10494_gb300 as pkg
    import workloads
    ctx = pkg.Context(0)
    if case in ("shared-dims", "perdesign-dims", "tps-timing"):
        run_timing_case(case, pkg, ctx)
        return
    if case == "tps":
        # two fits and one maximisation of the paper's 2000-point spline, k = 2
        rng = np.random.default_rng(2002)
        x = torch.as_tensor(rng.uniform(0, 1, (1, 2000, 2)), dtype=torch.float64, device="cuda")
        y = torch.as_tensor(rng.normal(0, 1, (1, 2000)), dtype=torch.float64, device="cuda")
        for _ in range(2):
            fit = pkg.mc_tps_fit(ctx, x, y, smoothing=0.01)
        pkg.mc_tps_argmax(ctx, x, fit, torch.zeros(2, dtype=torch.float64, device="cuda"),
                          torch.ones(2, dtype=torch.float64, device="cuda"), iters=300)
        ctx.sync_status()
        return
    if case in ("smooth", "smooth-f32"):
        S, G = 512, 256                       # FP64: 256 MB in, 256 MB out
        if case == "smooth-f32":
            S = 1024                          # FP32: 256 MB in, 256 MB out
        v = torch.rand(S * G * G, dtype=torch.float64 if case == "smooth" else torch.float32, device="cuda")
        for _ in range(3):
            pkg.mc_smooth_argmax(ctx, v, S, G, G, bandwidth=3.0, degree=2)
        ctx.sync_status()
        return
    if case in ("c2-shared", "c2-shared-full"):
        # two scenarios of the d=3 grid (2 x 4096 designs, one stream each),
        # or the whole grid of the timed step, 1e6 draws
        prob = workloads.c2(n_scen=2 if case == "c2-shared" else 16, n_draws=1_000_000)
        dp = pkg.DeviceProblem.from_workload(prob)
        jac = torch.as_tensor(prob.jac_packed(), dtype=torch.float64, device="cuda")
        fwd = pkg.Plan(ctx, dp, shared=True)
        adj = pkg.Plan(ctx, dp, shared=True, grad=True, k=4)
        for s in range(2):
            fwd.eval(s)
            adj.grad(s, jac, 0.01)
        ctx.sync_status()
        return
    if case == "c2-small":
        prob = workloads.c2(n_scen=2, g1=8, g2=8, n_draws=1_000_000)
    elif case == "c4-small":
        prob = workloads.c4(g1=4, g2=4, n_draws=10_000_000)
    else:
        prob = workloads.c5(g1=4, g2=4, n_draws=2_000_000)
    dp = pkg.DeviceProblem.from_workload(prob)
    jac = torch.as_tensor(prob.jac_packed(), dtype=torch.float64, device="cuda")
    fwd = pkg.Plan(ctx, dp)
    adj = pkg.Plan(ctx, dp, grad=True, k=4)
    for s in range(2):
        fwd.eval(s)
        adj.grad(s, jac, 0.01)
    ctx.sync_status()


def main():
    args = parse_args()
    if args.case:
        run_case(args.case)
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if args.impl == "ours" else "gloo")
    if args.impl == "reference":
        run_reference(args, rank)
    else:
        run_ours(args, rank, world)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
