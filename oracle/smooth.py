"""FP64 local-polynomial smoother and argmax over a design grid (oracle).

TEST INFRASTRUCTURE ONLY: imported by tests, never by the CUDA library.

Sec. 2.3 fits a smooth surface to the noisy Monte Carlo values P_hat(alpha)
on many design points and takes the point with the largest smoothed value as
the starting point of the Newton search.  The paper fits a thin-plate spline;
the engine uses local-polynomial regression over the regular design grid, and
this module is its plain definition:

  for each grid point (i, j) (coordinates in grid steps), minimise
      sum_{k,l} W_kl (P_hat_kl - beta . x_kl)^2
  over the points with positive weight, W_kl = w((k-i)/h) w((l-j)/h),
  tricube w(u) = (1 - |u|^3)^3 for |u| < 1; x_kl holds the monomials of
  (k-i, l-j) up to the degree ({1,x,y,x^2,xy,y^2} at degree 2); the smoothed
  value is beta_0.  A grid with one row (or column) uses the 1-D basis.
  Windows are cut at the grid edges.

The argmax is the lowest row-major index among the largest values.
"""
import numpy as np


def tricube(u):
    a = np.abs(u)
    return np.where(a < 1.0, (1.0 - a ** 3) ** 3, 0.0)


def _basis(dx, dy, degree, two_d):
    cols = [np.ones_like(dx)]
    if degree >= 1:
        cols.append(dx)
        if two_d:
            cols.append(dy)
    if degree >= 2:
        cols.append(dx * dx)
        if two_d:
            cols.append(dx * dy)
            cols.append(dy * dy)
    return np.stack(cols, axis=-1)


def smooth_grid(P, bandwidth=3.0, degree=2):
    """Smooth one G1 x G2 grid of values; returns the FP64 smoothed grid."""
    P = np.asarray(P, dtype=np.float64)
    G1, G2 = P.shape
    one_d = (G1 == 1) or (G2 == 1)
    vals = P.reshape(-1) if one_d else None
    out = np.empty_like(P)
    reach = int(np.ceil(bandwidth)) - 1 if float(bandwidth).is_integer() else int(np.floor(bandwidth))
    if one_d:
        n = vals.shape[0]
        for i in range(n):
            lo, hi = max(0, i - reach), min(n - 1, i + reach)
            k = np.arange(lo, hi + 1)
            dx = (k - i).astype(np.float64)
            W = tricube(dx / bandwidth)
            X = _basis(dx, None, degree, False)
            sw = np.sqrt(W)
            beta = np.linalg.lstsq(X * sw[:, None], vals[k] * sw, rcond=None)[0]
            out.reshape(-1)[i] = beta[0]
        return out
    for i in range(G1):
        for j in range(G2):
            ks = np.arange(max(0, i - reach), min(G1 - 1, i + reach) + 1)
            ls = np.arange(max(0, j - reach), min(G2 - 1, j + reach) + 1)
            K, Lg = np.meshgrid(ks, ls, indexing="ij")
            dx = (K - i).astype(np.float64).ravel()
            dy = (Lg - j).astype(np.float64).ravel()
            W = tricube(dx / bandwidth) * tricube(dy / bandwidth)
            X = _basis(dx, dy, degree, True)
            sw = np.sqrt(W)
            y = P[K.ravel(), Lg.ravel()]
            beta = np.linalg.lstsq(X * sw[:, None], y * sw, rcond=None)[0]
            out[i, j] = beta[0]
    return out


def argmax_lowest(values):
    """Index of the largest value, lowest row-major index on ties."""
    flat = np.asarray(values, dtype=np.float64).reshape(-1)
    return int(np.argmax(flat)), float(flat.max())


def smooth_argmax(P_all, G1, G2, bandwidth=3.0, degree=2):
    """Per scenario: smoothed grid, its argmax (index, value), raw argmax."""
    P_all = np.asarray(P_all, dtype=np.float64).reshape(-1, G1, G2)
    sm = np.stack([smooth_grid(P, bandwidth, degree) for P in P_all])
    arg = [argmax_lowest(s) for s in sm]
    raw = [argmax_lowest(P) for P in P_all]
    return sm, np.array([a[0] for a in arg]), np.array([a[1] for a in arg]), \
        np.array([r[0] for r in raw]), np.array([r[1] for r in raw])
