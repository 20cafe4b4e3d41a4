"""FP64 Monte Carlo oracle (Sec. 2.2, Eq. 5-7) -- ctypes wrapper of mc_oracle.c.

TEST INFRASTRUCTURE ONLY: imported by tests and by the CPU-baseline leg of
the benchmark, never by the CUDA library.

The estimator draws z ~ N(0, I) from the counter-based stream described in
mc_oracle.c, forms y = L z and counts draws with y_i > t_i for some i
(t = b - mu), i.e. draws of X = mu + L z that reject some hypothesis.
"""
import ctypes
import math
import os

import numpy as np

from . import build as _build

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        u64, i64, i32, f64 = ctypes.c_uint64, ctypes.c_int64, ctypes.c_int32, ctypes.c_double
        P = ctypes.POINTER
        L.oracle_philox4x32_10.argtypes = [P(ctypes.c_uint32), P(ctypes.c_uint32), P(ctypes.c_uint32)]
        L.oracle_philox_stream.argtypes = [u64, u64, u64, u64, P(ctypes.c_uint32)]
        L.oracle_normals.argtypes = [u64, u64, u64, u64, P(f64)]
        L.oracle_uniform.argtypes = [ctypes.c_uint32]
        L.oracle_uniform.restype = f64
        L.oracle_cholesky.argtypes = [ctypes.c_int, P(f64), P(f64)]
        L.oracle_cholesky.restype = ctypes.c_int
        L.oracle_mc_batch.argtypes = [i64, P(i32), P(f64), P(i64), P(f64), P(i64), u64,
                                      P(u64), P(u64), P(u64), f64, f64,
                                      P(u64), P(u64), P(f64), P(f64), P(f64)]
        L.oracle_num_threads.restype = ctypes.c_int
        L.oracle_set_num_threads.argtypes = [ctypes.c_int]
        L.oracle_set_num_threads.restype = None
        _lib = L
    return _lib


def _ptr(a, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def philox4x32_10(counter, key):
    """One Philox4x32-10 block: counter (4 u32), key (2 u32) -> 4 u32."""
    c = np.ascontiguousarray(counter, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().oracle_philox4x32_10(_ptr(c, ctypes.c_uint32), _ptr(k, ctypes.c_uint32), _ptr(out, ctypes.c_uint32))
    return out


def philox_stream(seed, key, call_begin, count):
    out = np.zeros(4 * count, dtype=np.uint32)
    lib().oracle_philox_stream(seed, key, call_begin, count, _ptr(out, ctypes.c_uint32))
    return out


def uniform(word):
    return lib().oracle_uniform(int(word))


def normals(seed, key, m_begin, count):
    """Normals number m_begin .. m_begin+count-1 of stream (seed, key), FP64."""
    out = np.zeros(count, dtype=np.float64)
    lib().oracle_normals(seed, key, m_begin, count, _ptr(out, ctypes.c_double))
    return out


def cholesky(Sigma):
    """Lower Cholesky factor (textbook algorithm in C); raises on a non-SPD pivot."""
    S = np.ascontiguousarray(Sigma, dtype=np.float64)
    d = S.shape[0]
    L = np.zeros((d, d))
    rc = lib().oracle_cholesky(d, _ptr(S, ctypes.c_double), _ptr(L, ctypes.c_double))
    if rc != 0:
        raise np.linalg.LinAlgError("pivot %d is not positive" % (rc - 1))
    return L


def mc_batch(designs, seed, eps=0.0, h=0.0, grad=False):
    """Run the FP64 estimator on a list of designs.

    designs: list of dicts with keys
        Sigma (d x d), t (d,), key (u64), n_draws (u64), draw_begin (u64, optional)
    Returns dict of arrays: hits, ambiguous, and (grad) A, B, G lists of (d,) arrays.
    """
    J = len(designs)
    ds = np.array([len(x["t"]) for x in designs], dtype=np.int32)
    L_blocks, L_off, t_off = [], np.zeros(J, np.int64), np.zeros(J, np.int64)
    off_L = off_t = 0
    chol_cache = {}
    for j, x in enumerate(designs):
        sig = np.ascontiguousarray(x["Sigma"], dtype=np.float64)
        ck = sig.tobytes()
        if ck not in chol_cache:
            chol_cache[ck] = cholesky(sig)
        L_blocks.append(chol_cache[ck].ravel())
        L_off[j], t_off[j] = off_L, off_t
        off_L += ds[j] * ds[j]
        off_t += ds[j]
    Lcat = np.ascontiguousarray(np.concatenate(L_blocks) if J else np.zeros(1))
    tcat = np.ascontiguousarray(np.concatenate([np.asarray(x["t"], np.float64) for x in designs]) if J else np.zeros(1))
    keys = np.array([x["key"] for x in designs], dtype=np.uint64)
    n = np.array([x["n_draws"] for x in designs], dtype=np.uint64)
    begin = np.array([x.get("draw_begin", 0) for x in designs], dtype=np.uint64)
    hits = np.zeros(J, np.uint64)
    amb = np.zeros(J, np.uint64)
    A = np.zeros(max(off_t, 1)); B = np.zeros(max(off_t, 1)); G = np.zeros(max(off_t, 1))
    nullp = ctypes.POINTER(ctypes.c_double)()
    lib().oracle_mc_batch(J, _ptr(ds, ctypes.c_int32), _ptr(Lcat, ctypes.c_double), _ptr(L_off, ctypes.c_int64),
                          _ptr(tcat, ctypes.c_double), _ptr(t_off, ctypes.c_int64), seed,
                          _ptr(keys, ctypes.c_uint64), _ptr(begin, ctypes.c_uint64), _ptr(n, ctypes.c_uint64),
                          eps, h, _ptr(hits, ctypes.c_uint64), _ptr(amb, ctypes.c_uint64),
                          _ptr(A, ctypes.c_double) if grad else nullp,
                          _ptr(B, ctypes.c_double) if grad else nullp,
                          _ptr(G, ctypes.c_double) if (grad and h > 0) else nullp)
    out = {"hits": hits, "ambiguous": amb}
    if grad:
        out["A"] = [A[t_off[j]:t_off[j] + ds[j]].copy() for j in range(J)]
        out["B"] = [B[t_off[j]:t_off[j] + ds[j]].copy() for j in range(J)]
        out["G"] = [G[t_off[j]:t_off[j] + ds[j]].copy() for j in range(J)]
    return out


def lr_gradient_mu(Sigma, A, B, hits, n):
    """d p / d mu by the likelihood ratio with the z control variate:
    grad_mu p = L^{-T} (A - p_hat B) / N, because grad_mu log f(X) = Sigma^{-1}(X - mu)
    = L^{-T} z and E[z] = 0."""
    L = cholesky(Sigma)
    p = float(hits) / float(n)
    v = (np.asarray(A) - p * np.asarray(B)) / float(n)
    return np.linalg.solve(L.T, v)


def num_threads():
    return lib().oracle_num_threads()


def set_num_threads(n):
    """Threads of mc_batch's loop over designs from now on (OpenMP)."""
    lib().oracle_set_num_threads(int(n))


def se_binomial(p, n):
    return math.sqrt(max(p * (1.0 - p), 0.0) / n)


__all__ = ["philox4x32_10", "philox_stream", "uniform", "normals", "cholesky", "mc_batch",
           "lr_gradient_mu", "num_threads", "set_num_threads", "se_binomial", "os"]
