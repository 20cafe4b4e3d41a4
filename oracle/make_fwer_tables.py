"""Write workloads/fwer_tables.json: calibrated alpha scales s(a) (Eq. 2).

TEST INFRASTRUCTURE: this script calls only the oracle (and reads scenario
parameters from the seeded input module).  For each benchmark scenario and
each allocation a on a fine grid it solves

    1 - Phi_Sigma(Z_{1 - s w_1(a)}, ..., Z_{1 - s w_d(a)}) = alpha_0 = 0.025

for s by Brent's method on the oracle's quadrature (tolerance 1e-13 in the
FWER, 1e-15 in s).  The input module interpolates s(a) with a cubic spline.

Usage: python -m oracle.make_fwer_tables
"""
import json
import multiprocessing as mp
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
sys.path.insert(0, ROOT)

from oracle import quad  # noqa: E402
import workloads  # noqa: E402

N_A = 129
A_GRID = np.linspace(workloads.A_RANGE[0], workloads.A_RANGE[1], N_A)


def weights(a, d):
    w = np.full(d, a / (d - 1))
    w[0] = 1.0 - a
    return w


def _solve(args):
    a, d, structure = args
    Sigma = quad.structured_sigma(d, structure)
    return quad.calibrate_scale(weights(a, d), workloads.ALPHA0, Sigma, structure)


def curve(pool, d, structure):
    return [float(x) for x in pool.map(_solve, [(float(a), d, structure) for a in A_GRID])]


def main():
    t0 = time.time()
    ctx = mp.get_context("spawn")
    out = {"alpha0": workloads.ALPHA0, "note": "alpha scale s(a) solving the FWER constraint (Eq. 2)"}
    with ctx.Pool(os.cpu_count()) as pool:
        eq = {"kind": "equi", "rho": 0.5}
        out["c1"] = {"rho": 0.5, "d": 3,
                     "scale": quad.calibrate_scale(np.ones(3) / 3, workloads.ALPHA0,
                                                   quad.structured_sigma(3, eq), eq)}
        scen = []
        for dp, dm, rho in workloads.c2_scenarios(16):
            st = {"kind": "equi", "rho": rho}
            scen.append({"rho": rho, "a": [float(a) for a in A_GRID], "scale": curve(pool, 3, st)})
        out["c2"] = {"scenarios": scen}
        st = {"kind": "ar1", "rho": 0.3}
        out["c4"] = {"rho": 0.3, "d": 10, "a": [float(a) for a in A_GRID], "scale": curve(pool, 10, st)}
        st = {"kind": "block", "sizes": [5, 5, 5, 5], "rho_in": 0.6, "rho_out": 0.1}
        out["c5"] = {"sizes": [5, 5, 5, 5], "rho_in": 0.6, "rho_out": 0.1, "d": 20,
                     "a": [float(a) for a in A_GRID], "scale": curve(pool, 20, st)}
    with open(workloads.TABLE_PATH, "w") as f:
        json.dump(out, f, indent=1)
    print("wrote %s in %.1f s" % (workloads.TABLE_PATH, time.time() - t0))


if __name__ == "__main__":
    main()
