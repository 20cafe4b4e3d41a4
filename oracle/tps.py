"""Thin-plate spline smoothing and its maximiser (oracle, test infrastructure).

TEST INFRASTRUCTURE ONLY: used by tests; nothing in the CUDA library
imports this module.

Sec. 2.3 fits a thin-plate spline (TPS) to the N3 noisy estimates P_hat(alpha)
and maximises the fitted surface with a quasi-Newton method started at the
best fitted point.  For points x_i in R^k (k = 1, 2, 3) and values y_i the
smoothing spline with parameter s >= 0 is

    f(x) = sum_i c_i eta(|x - x_i|) + d_0 + sum_j d_j x_j,
    [K + s I   P] [c]   [y]
    [P^T       0] [d] = [0],    K_ij = eta(|x_i - x_j|),  P = [1, x],

with the radial function of the second-order spline in k dimensions
(Green & Silverman, Ch. 7): eta(r) = r^3 (k = 1), r^2 log r (k = 2),
-r (k = 3); s = 0 interpolates.  The linear system is solved directly
(numpy's dense solver, a library step); the fitted values at the data are
y - s c.
"""
import numpy as np
from scipy import optimize


def eta(r, k):
    r = np.asarray(r, dtype=np.float64)
    if k == 1:
        return r ** 3
    if k == 2:
        with np.errstate(divide="ignore", invalid="ignore"):
            return np.where(r > 0, r * r * np.log(np.where(r > 0, r, 1.0)), 0.0)
    if k == 3:
        return -r
    raise ValueError("k must be 1, 2 or 3")


def _dist(a, b):
    return np.sqrt(((a[:, None, :] - b[None, :, :]) ** 2).sum(-1))


def fit(x, y, s=0.0):
    """Coefficients (c[N], d[k + 1]) of the smoothing spline."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    N, k = x.shape
    K = eta(_dist(x, x), k)
    P = np.hstack([np.ones((N, 1)), x])
    m = k + 1
    M = np.zeros((N + m, N + m))
    M[:N, :N] = K + s * np.eye(N)
    M[:N, N:] = P
    M[N:, :N] = P.T
    sol = np.linalg.solve(M, np.concatenate([y, np.zeros(m)]))
    return sol[:N], sol[N:]


def evaluate(xq, x, c, d):
    xq = np.atleast_2d(np.asarray(xq, dtype=np.float64))
    k = x.shape[1]
    return eta(_dist(xq, x), k) @ c + d[0] + xq @ d[1:]


def gradient(xq, x, c, d):
    """Gradient of f at one point xq (k,)."""
    xq = np.asarray(xq, dtype=np.float64)
    k = x.shape[1]
    diff = xq[None, :] - x
    r = np.sqrt((diff ** 2).sum(-1))
    if k == 1:
        g = (3.0 * r)[:, None] * diff                    # d(r^3) = 3 r^2 dr, dr = diff / r
    elif k == 2:
        with np.errstate(divide="ignore", invalid="ignore"):
            fac = np.where(r > 0, 2.0 * np.log(np.where(r > 0, r, 1.0)) + 1.0, 0.0)   # eta'(r) / r
        g = fac[:, None] * diff
    else:
        with np.errstate(divide="ignore", invalid="ignore"):
            fac = np.where(r > 0, -1.0 / np.where(r > 0, r, 1.0), 0.0)
        g = fac[:, None] * diff
    return c @ g + d[1:]


def argmax(x, c, d, lo, hi, x0=None):
    """Maximiser of the fitted surface in the box [lo, hi] by L-BFGS-B
    (scipy), started at the data point with the largest fitted value
    unless x0 is given."""
    x = np.asarray(x, dtype=np.float64)
    if x0 is None:
        inside = np.all((x >= lo) & (x <= hi), axis=1)
        fv = evaluate(x, x, c, d)
        fv[~inside] = -np.inf
        x0 = x[int(np.argmax(fv))]
    res = optimize.minimize(lambda z: -evaluate(z, x, c, d)[0], x0, jac=lambda z: -gradient(z, x, c, d),
                            method="L-BFGS-B", bounds=list(zip(lo, hi)),
                            options={"ftol": 1e-15, "gtol": 1e-12, "maxiter": 500})
    return res.x, -res.fun


def gcv(x, y, s):
    """Generalised cross-validation score of the smoothing spline,
    V(s) = N |(I - A_s) y|^2 / tr(I - A_s)^2 with A_s the influence matrix
    (fitted = A_s y), through the inverse of the full system: the block G
    with c = G y gives (I - A_s) y = s c and tr(I - A_s) = s tr G."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    N, k = x.shape
    K = eta(_dist(x, x), k)
    P = np.hstack([np.ones((N, 1)), x])
    m = k + 1
    M = np.zeros((N + m, N + m))
    M[:N, :N] = K + s * np.eye(N)
    M[:N, N:] = P
    M[N:, :N] = P.T
    G = np.linalg.inv(M)[:N, :N]
    c = G @ y
    return N * float((s * c) @ (s * c)) / float(s * np.trace(G)) ** 2
