"""ctypes binding of libmcdesign (include/mcdesign.h): argument marshalling only.

Every computation runs in the CUDA library; this module turns torch tensors
into device pointers and numpy arrays into host pointers, checks return
codes and raises.  There is no CPU fallback: without the built library or a
CUDA device the calls raise.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libmcdesign.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "mcdesign.h")

MCD_OK, MCD_EINVAL, MCD_ENOTSPD, MCD_ECUDA, MCD_ENOMEM, MCD_EUNSUPPORTED, MCD_ENAN = 0, 1, 2, 3, 5, 6, 7
MCD_ANY_EXCEEDS, MCD_ALL_BELOW = 0, 1
MCD_PLAN_GRAD, MCD_PLAN_AUTOTUNE, MCD_PLAN_GRAPH, MCD_PLAN_FP64, MCD_PLAN_TIMING, MCD_PLAN_SHARED = 1, 2, 4, 8, 16, 32
MCD_SHARED_MIN = 32
# instruction classes of mcd_pipe_rate, in MCD_PIPE_* order
PIPE_CLASSES = ("mul_wide", "mad_lo", "lop3", "ffma", "lg2", "sqrt", "sin", "cos", "ex2", "rcp", "mixed", "lds128", "philox",
                "ffma2")
MCD_MAX_D = 20

_c_i32p = ctypes.POINTER(ctypes.c_int32)
_c_u64p = ctypes.POINTER(ctypes.c_uint64)


class CProblem(ctypes.Structure):
    _fields_ = [("n_scen", ctypes.c_int32), ("n_design", ctypes.c_int32),
                ("scen_d", _c_i32p), ("design_scen", _c_i32p), ("n_draws", _c_u64p),
                ("draw_begin", _c_u64p), ("key", _c_u64p),
                ("Sigma", ctypes.c_void_p), ("mu", ctypes.c_void_p), ("b", ctypes.c_void_p),
                ("region", ctypes.c_int32)]


class MCDError(RuntimeError):
    def __init__(self, code, msg, index=-1):
        super().__init__("mcdesign error %d: %s%s" % (code, msg, "" if index < 0 else " (index %d)" % index))
        self.code = code
        self.index = index


_lib = None


def load(path=LIB_PATH):
    """Load libmcdesign.so (raises when it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("libmcdesign.so is not built (%s); run paper_2005_10494_gb300/build.py" % path)
    L = ctypes.CDLL(path)
    vp, i32, i64, u64, f64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
    sig = {
        "mcd_create": (i32, [ctypes.POINTER(vp), ctypes.c_int]),
        "mcd_destroy": (None, [vp]),
        "mcd_last_error": (ctypes.c_char_p, [vp]),
        "mcd_error_index": (i64, [vp]),
        "mcd_sync_status": (i32, [vp, vp]),
        "mcd_plan_create": (i32, [vp, ctypes.POINTER(CProblem), i32, i32, ctypes.POINTER(vp)]),
        "mcd_plan_destroy": (None, [vp]),
        "mcd_plan_eval": (i32, [vp, u64, vp, vp, vp, vp]),
        "mcd_plan_grad": (i32, [vp, u64, vp, f64, vp, vp, vp, vp, vp, vp]),
        "mcd_plan_config": (i32, [vp, i32, ctypes.POINTER(i32), ctypes.POINTER(i64), ctypes.POINTER(i32)]),
        "mcd_plan_tiles": (i64, [vp]),
        "mcd_plan_kernel_ms": (i32, [vp, ctypes.POINTER(ctypes.c_float)]),
        "mc_design_eval": (i32, [vp, ctypes.POINTER(CProblem), u64, vp, vp, vp, vp]),
        "mc_design_grad": (i32, [vp, ctypes.POINTER(CProblem), u64, i32, vp, f64, vp, vp, vp, vp, vp, vp]),
        "mc_smooth_argmax": (i32, [vp, i32, i32, i32, vp, f64, i32, vp, vp, vp, vp, vp, vp]),
        "mc_smooth_argmax_f32": (i32, [vp, i32, i32, i32, vp, f64, i32, vp, vp, vp, vp, vp, vp]),
        "mc_fwer_calibrate": (i32, [vp, ctypes.POINTER(CProblem), vp, f64, i32, u64, vp, vp, vp, vp]),
        "mc_tps_fit": (i32, [vp, i32, i32, i32, vp, vp, f64, vp, vp, vp]),
        "mc_tps_argmax": (i32, [vp, i32, i32, i32, vp, vp, vp, vp, vp, i32, vp, vp, vp]),
        "mc_tps_gcv": (i32, [vp, i32, i32, vp, vp, i32, ctypes.POINTER(f64), vp, vp]),
        "mcd_debug_normals": (i32, [vp, u64, u64, u64, u64, vp, vp, vp, vp]),
        "mc_design_eval_noalloc": (i32, [ctypes.c_int, ctypes.POINTER(CProblem), u64, vp, vp, vp, vp]),
        "mcd_pipe_rate": (i32, [vp, i32, i32, ctypes.POINTER(f64), vp]),
        "mcd_debug_fail_next": (i32, [vp, i32]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("mcdesign needs a CUDA device; none is available")
    return torch


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


class Context:
    """A library context on one CUDA device (mcd_create / mcd_destroy)."""

    def __init__(self, device=0):
        _torch()
        self.lib = load()
        self.device = device
        h = ctypes.c_void_p()
        rc = self.lib.mcd_create(ctypes.byref(h), device)
        if rc != MCD_OK:
            raise MCDError(rc, "mcd_create failed on device %d" % device)
        self.handle = h

    def check(self, rc):
        if rc != MCD_OK:
            msg = self.lib.mcd_last_error(self.handle).decode()
            raise MCDError(rc, msg, self.lib.mcd_error_index(self.handle))

    def sync_status(self, stream=None):
        """Wait for the stream and raise on a device-side error (non-SPD, NaN)."""
        self.check(self.lib.mcd_sync_status(self.handle, _stream(stream)))

    def fail_next_launch(self, cuda_error):
        """Host-side fault injection (mcd_debug_fail_next): the next plan
        launch on this context returns MCD_ECUDA without queuing work."""
        self.check(self.lib.mcd_debug_fail_next(self.handle, int(cuda_error)))

    def close(self):
        if getattr(self, "handle", None):
            self.lib.mcd_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class DeviceProblem:
    """A batch of designs: host metadata plus device Sigma, mu, b (torch, FP64).

    scen_d[S], design_scen[J], n_draws[J], key[J], draw_begin[J] are numpy
    arrays; Sigma is the packed row-major d_s x d_s blocks, mu and b the
    packed d values of each design, all torch.float64 CUDA tensors.
    """

    def __init__(self, scen_d, design_scen, n_draws, key, Sigma, mu, b, draw_begin=None,
                 region=MCD_ANY_EXCEEDS):
        self.scen_d = np.ascontiguousarray(scen_d, dtype=np.int32)
        self.design_scen = np.ascontiguousarray(design_scen, dtype=np.int32)
        self.n_draws = np.ascontiguousarray(n_draws, dtype=np.uint64)
        self.key = np.ascontiguousarray(key, dtype=np.uint64)
        self.draw_begin = None if draw_begin is None else np.ascontiguousarray(draw_begin, dtype=np.uint64)
        self.Sigma, self.mu, self.b = Sigma, mu, b
        for t in (Sigma, mu, b):
            if not (t.is_cuda and t.is_contiguous()) or str(t.dtype) != "torch.float64":
                raise ValueError("Sigma, mu, b must be contiguous float64 CUDA tensors")
        self.region = region
        J = self.design_scen.shape[0]
        self.n_scen, self.n_design = int(self.scen_d.shape[0]), int(J)
        d = self.scen_d[self.design_scen] if J else np.zeros(0, np.int32)
        self.design_d = d
        self.vec_off = np.concatenate([[0], np.cumsum(d)[:-1]]).astype(np.int64) if J else np.zeros(0, np.int64)
        self.vec_len = int(d.sum()) if J else 0
        self.c = CProblem(self.n_scen, self.n_design,
                          self.scen_d.ctypes.data_as(_c_i32p), self.design_scen.ctypes.data_as(_c_i32p),
                          self.n_draws.ctypes.data_as(_c_u64p),
                          None if self.draw_begin is None else self.draw_begin.ctypes.data_as(_c_u64p),
                          self.key.ctypes.data_as(_c_u64p),
                          Sigma.data_ptr(), mu.data_ptr(), b.data_ptr(), region)

    @classmethod
    def from_workload(cls, prob, device="cuda", region=MCD_ANY_EXCEEDS):
        """Upload a workloads.Problem (host numpy) to the device."""
        torch = _torch()
        f64 = torch.float64
        Sigma = torch.as_tensor(prob.sigma_packed(), dtype=f64).to(device).contiguous()
        mu = torch.as_tensor(prob.mu_packed(), dtype=f64).to(device).contiguous()
        b = torch.as_tensor(prob.b_packed(), dtype=f64).to(device).contiguous()
        if mu.numel() == 0:
            mu = torch.zeros(1, dtype=f64, device=device)
            b = torch.zeros(1, dtype=f64, device=device)
        return cls(prob.scen_d, prob.design_scen, prob.n_draws, prob.keys, Sigma, mu, b,
                   draw_begin=prob.draw_begin, region=region)


def _outputs(J, vec_len, k, grad, device, want_sig):
    """Output buffers of one call kind: exactly the arrays that call writes."""
    torch = _torch()
    out = {"hits": torch.empty(max(J, 1), dtype=torch.int64, device=device),
           "p": torch.empty(max(J, 1), dtype=torch.float64, device=device)}
    if not grad:
        out["se"] = torch.empty(max(J, 1), dtype=torch.float64, device=device)
    else:
        n = J * k if k > 0 else vec_len
        out["grad_lr"] = torch.empty(max(n, 1), dtype=torch.float64, device=device)
        out["grad_se"] = torch.empty(max(n, 1), dtype=torch.float64, device=device)
        if want_sig:
            out["grad_sig"] = torch.empty(max(n, 1), dtype=torch.float64, device=device)
    return out


def _trim(out, J, n):
    res = {}
    for name, t in out.items():
        res[name] = t[:J] if name in ("hits", "p", "se") else t[:n]
    return res


class Plan:
    """mcd_plan_create / mcd_plan_eval / mcd_plan_grad."""

    def __init__(self, ctx, prob, grad=False, k=0, autotune=False, graph=False, fp64=False, timing=False,
                 shared=False):
        self.ctx, self.prob, self.k = ctx, prob, k
        flags = (MCD_PLAN_GRAD if grad else 0) | (MCD_PLAN_AUTOTUNE if autotune else 0) \
            | (MCD_PLAN_GRAPH if graph else 0) | (MCD_PLAN_FP64 if fp64 else 0) | (MCD_PLAN_TIMING if timing else 0) \
            | (MCD_PLAN_SHARED if shared else 0)
        h = ctypes.c_void_p()
        ctx.check(ctx.lib.mcd_plan_create(ctx.handle, ctypes.byref(prob.c), flags, k, ctypes.byref(h)))
        self.handle = h
        self._out = {}

    def tiles(self):
        return int(self.ctx.lib.mcd_plan_tiles(self.handle))

    def kernel_ms(self):
        """Duration of the sampling kernels of the last launch (timing plans)."""
        ms = ctypes.c_float()
        self.ctx.check(self.ctx.lib.mcd_plan_kernel_ms(self.handle, ctypes.byref(ms)))
        return float(ms.value)

    def config(self, d):
        th, bps = ctypes.c_int32(), ctypes.c_int32()
        td = ctypes.c_int64()
        self.ctx.check(self.ctx.lib.mcd_plan_config(self.handle, d, ctypes.byref(th), ctypes.byref(td),
                                                     ctypes.byref(bps)))
        return {"threads": th.value, "tile_draws": td.value, "blocks_per_sm": bps.value}

    def _buffers(self, grad, want_sig):
        key = (grad, want_sig)
        if key not in self._out:
            self._out[key] = _outputs(self.prob.n_design, self.prob.vec_len, self.k, grad,
                                      self.prob.Sigma.device, want_sig)
        return self._out[key]

    def eval(self, seed, stream=None, out=None):
        """Queue an evaluation; returns dict hits, p, se (device tensors, reused
        by the next call of the same kind unless `out` is given)."""
        o = out or self._buffers(False, False)
        self.ctx.check(self.ctx.lib.mcd_plan_eval(self.handle, seed, _ptr(o["hits"]), _ptr(o["p"]),
                                                  _ptr(o["se"]), _stream(stream)))
        return _trim(o, self.prob.n_design, 0)

    def grad(self, seed, jac=None, h=0.0, stream=None, out=None):
        """Queue estimate + derivatives; jac: [sum_j d_j * k] FP64 CUDA tensor or None."""
        o = out or self._buffers(True, h > 0)
        n = self.prob.n_design * self.k if self.k > 0 else self.prob.vec_len
        self.ctx.check(self.ctx.lib.mcd_plan_grad(self.handle, seed, _ptr(jac), float(h), _ptr(o["hits"]),
                                                  _ptr(o["p"]), _ptr(o["grad_lr"]), _ptr(o.get("grad_sig")),
                                                  _ptr(o["grad_se"]), _stream(stream)))
        return _trim(o, self.prob.n_design, n)

    def close(self):
        if getattr(self, "handle", None):
            self.ctx.lib.mcd_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mc_design_eval(ctx, prob, seed, stream=None):
    """One-shot estimate of p for every design (plan, launch, release)."""
    o = _outputs(prob.n_design, prob.vec_len, 0, False, prob.Sigma.device, False)
    ctx.check(ctx.lib.mc_design_eval(ctx.handle, ctypes.byref(prob.c), seed, _ptr(o["hits"]), _ptr(o["p"]),
                                     _ptr(o["se"]), _stream(stream)))
    return _trim(o, prob.n_design, 0)


def mc_design_eval_noalloc(prob, seed, device=0, stream=None, out=None):
    """mc_design_eval for callers that cannot allocate device memory: one
    scenario, equal draw counts, at most 16384 designs; the library's static
    scratch array is shared by all calls (serialise overlapping calls).  Pass
    preallocated `out` tensors (hits int64, p, se float64) to allocate nothing."""
    lib = load()
    o = out or _outputs(prob.n_design, prob.vec_len, 0, False, prob.Sigma.device, False)
    rc = lib.mc_design_eval_noalloc(device, ctypes.byref(prob.c), seed, _ptr(o["hits"]), _ptr(o["p"]),
                                    _ptr(o["se"]), _stream(stream))
    if rc != MCD_OK:
        raise MCDError(rc, "mc_design_eval_noalloc rejected the call")
    return _trim(o, prob.n_design, 0)


def mc_design_grad(ctx, prob, seed, k=0, jac=None, h=0.0, stream=None):
    """One-shot estimate of p and its derivatives."""
    o = _outputs(prob.n_design, prob.vec_len, k, True, prob.Sigma.device, h > 0)
    n = prob.n_design * k if k > 0 else prob.vec_len
    ctx.check(ctx.lib.mc_design_grad(ctx.handle, ctypes.byref(prob.c), seed, k, _ptr(jac), float(h),
                                     _ptr(o["hits"]), _ptr(o["p"]), _ptr(o["grad_lr"]), _ptr(o.get("grad_sig")),
                                     _ptr(o["grad_se"]), _stream(stream)))
    return _trim(o, prob.n_design, n)


def mc_fwer_calibrate(ctx, prob, w, alpha0=0.025, rounds=14, seed=0, stream=None):
    """Scale of each design's alpha split w (FP64 CUDA tensor, layout of mu)
    such that the Monte Carlo FWER under mu = 0 equals alpha0 (Eq. 2);
    prob.mu and prob.b are not read.  Returns dict scale[J], b[sum d],
    fwer[J] (device tensors)."""
    torch = _torch()
    dev = prob.Sigma.device
    out = {"scale": torch.empty(max(prob.n_design, 1), dtype=torch.float64, device=dev),
           "b": torch.empty(max(prob.vec_len, 1), dtype=torch.float64, device=dev),
           "fwer": torch.empty(max(prob.n_design, 1), dtype=torch.float64, device=dev)}
    ctx.check(ctx.lib.mc_fwer_calibrate(ctx.handle, ctypes.byref(prob.c), _ptr(w), float(alpha0), int(rounds), seed,
                                        _ptr(out["scale"]), _ptr(out["b"]), _ptr(out["fwer"]), _stream(stream)))
    return {"scale": out["scale"][:prob.n_design], "b": out["b"][:prob.vec_len], "fwer": out["fwer"][:prob.n_design]}


def mc_tps_fit(ctx, x, y, smoothing=0.0, stream=None):
    """Thin-plate smoothing splines of n_surf surfaces: x [n_surf, n_pts, k]
    and y [n_surf, n_pts] FP64 CUDA tensors.  Returns dict coef
    [n_surf, n_pts + k + 1] (c then d) and fitted [n_surf, n_pts]."""
    torch = _torch()
    if x.dim() != 3 or y.dim() != 2 or x.shape[:2] != y.shape:
        raise ValueError("x must be [n_surf, n_pts, k] and y [n_surf, n_pts]")
    S, N, k = (int(v) for v in x.shape)
    x, y = x.contiguous(), y.contiguous()
    coef = torch.empty((S, N + k + 1), dtype=torch.float64, device=x.device)
    fitted = torch.empty((S, N), dtype=torch.float64, device=x.device)
    ctx.check(ctx.lib.mc_tps_fit(ctx.handle, S, N, k, _ptr(x), _ptr(y), float(smoothing), _ptr(coef), _ptr(fitted),
                                 _stream(stream)))
    return {"coef": coef, "fitted": fitted}


def mc_tps_gcv(ctx, x, y, s_values, stream=None):
    """GCV scores of the smoothing spline of one surface (x [n_pts, k],
    y [n_pts], FP64 CUDA tensors) for each smoothing value (host sequence).
    Returns an FP64 CUDA tensor [len(s_values)]."""
    torch = _torch()
    if x.dim() != 2 or y.dim() != 1 or x.shape[0] != y.shape[0]:
        raise ValueError("x must be [n_pts, k] and y [n_pts]")
    N, k = (int(v) for v in x.shape)
    sv = np.ascontiguousarray(s_values, dtype=np.float64)
    score = torch.empty(len(sv), dtype=torch.float64, device=x.device)
    ctx.check(ctx.lib.mc_tps_gcv(ctx.handle, N, k, _ptr(x.contiguous()), _ptr(y.contiguous()), len(sv),
                                 sv.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), _ptr(score), _stream(stream)))
    return score


def mc_tps_argmax(ctx, x, fit, lo, hi, iters=200, stream=None):
    """Maximiser of each fitted spline (mc_tps_fit's output `fit`) in the box
    [lo, hi] (FP64 CUDA tensors of k values).  Returns dict x [n_surf, k],
    f [n_surf]."""
    torch = _torch()
    S, N, k = (int(v) for v in x.shape)
    xb = torch.empty((S, k), dtype=torch.float64, device=x.device)
    fb = torch.empty(S, dtype=torch.float64, device=x.device)
    ctx.check(ctx.lib.mc_tps_argmax(ctx.handle, S, N, k, _ptr(x.contiguous()), _ptr(fit["coef"]), _ptr(fit["fitted"]),
                                    _ptr(lo.contiguous()), _ptr(hi.contiguous()), int(iters), _ptr(xb), _ptr(fb),
                                    _stream(stream)))
    return {"x": xb, "f": fb}


def mc_smooth_argmax(ctx, values, n_scen, g1, g2, bandwidth=3.0, degree=2, stream=None, smoothed=True,
                     raw=False):
    """Smooth n_scen grids of g1 x g2 values (an FP64 CUDA tensor:
    mc_smooth_argmax; FP32: mc_smooth_argmax_f32, outputs FP32) and take
    argmaxes; raw=True also returns the argmax of the unsmoothed values."""
    torch = _torch()
    dev = values.device
    if values.dtype == torch.float32:
        fn, ft = ctx.lib.mc_smooth_argmax_f32, torch.float32
    elif values.dtype == torch.float64:
        fn, ft = ctx.lib.mc_smooth_argmax, torch.float64
    else:
        raise TypeError("values must be float64 or float32")
    sm = torch.empty(n_scen * g1 * g2, dtype=ft, device=dev) if smoothed else None
    idx = torch.empty(n_scen, dtype=torch.int64, device=dev)
    val = torch.empty(n_scen, dtype=ft, device=dev)
    ridx = torch.empty(n_scen, dtype=torch.int64, device=dev) if raw else None
    rval = torch.empty(n_scen, dtype=ft, device=dev) if raw else None
    ctx.check(fn(ctx.handle, n_scen, g1, g2, _ptr(values), float(bandwidth), degree,
                 _ptr(sm), _ptr(idx), _ptr(val), _ptr(ridx), _ptr(rval), _stream(stream)))
    return {"smoothed": sm, "argmax_idx": idx, "argmax_val": val, "raw_idx": ridx, "raw_val": rval}


def debug_normals(ctx, seed, key, m_begin, count, stream=None):
    """Normals m_begin.. of stream (seed, key) from the kernels' FP32 and FP64
    paths, plus the raw Philox words of the calls they come from."""
    torch = _torch()
    z32 = torch.empty(max(count, 1), dtype=torch.float32, device="cuda")
    z64 = torch.empty(max(count, 1), dtype=torch.float64, device="cuda")
    ncalls = ((m_begin + count - 1) >> 2) - (m_begin >> 2) + 1 if count else 0
    words = torch.empty(max(4 * ncalls, 1), dtype=torch.int32, device="cuda")
    ctx.check(ctx.lib.mcd_debug_normals(ctx.handle, seed, key, m_begin, count, _ptr(z32), _ptr(z64),
                                        _ptr(words), _stream(stream)))
    return z32[:count], z64[:count], words[:4 * ncalls]


def pipe_rates(ctx, iters=4096, classes=PIPE_CLASSES, stream=None):
    """Operations per SM clock of each instruction class (mcd_pipe_rate)."""
    out = {}
    for name in classes:
        r = ctypes.c_double(0.0)
        ctx.check(ctx.lib.mcd_pipe_rate(ctx.handle, PIPE_CLASSES.index(name), int(iters), ctypes.byref(r),
                                        _stream(stream)))
        out[name] = r.value
    return out
