"""Write tests/golden/drops256_walls_z.json from a full FP64 CPU-oracle solve of
the 256^3 drop field (periodic x, y; walls z; rho 1000/1; dt = 1e-4).

Calls only the oracle and the seeded input generator.  Stored: a checksum of
the volume fraction (so a test can confirm it regenerates the same input), the
oracle's CG iteration count and residuals, its Lanczos eigenvalue estimates,
the error bound they give for the oracle's own p, and p and the corrected
velocity at seeded sample points.
Run:  python tests/golden/make_drops256_golden.py  (about 10-20 minutes).
"""
import hashlib
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)
import oracle  # noqa: E402
import paris_inputs as pi  # noqa: E402


def oracle_error_bound(res, b0):
    """Error bound of the oracle's own p from its final residual (Eq. poisson).

    The oracle solves A x = -b0 with A = -L symmetric positive definite on the
    mean-free space, so the error e = x - x_exact obeys
    ||e||_inf <= ||e||_2 <= ||r||_2 / lambda_min, ||r||_2 = rel_res_l2 ||b0||_2.
    lambda_min is the smallest Ritz value of the CG run's Lanczos tridiagonal,
    which lies at or above the true smallest non-zero eigenvalue, so the bound
    is an estimate, sharp once that Ritz value has converged.  The velocity
    error on a face is dt beta_f (e_R - e_L)/h <= 2 dt max(beta) ||e||_inf / h.
    """
    lmin, lmax = res.cg.lanczos_extremes()
    r2 = res.cg.rel_res_l2 * float(np.linalg.norm(b0.ravel()))
    e_inf = r2 / lmin
    p_inf = float(np.abs(res.p).max())
    beta_max = max(float(np.abs(b).max()) for b in res.beta)
    return {
        "lanczos_lambda_min": lmin, "lanczos_lambda_max": lmax,
        "kappa_estimate": lmax / lmin,
        "b_l2": float(np.linalg.norm(b0.ravel())),
        "p_err_inf_bound": e_inf,
        "p_rel_err_bound": e_inf / p_inf,
        "u_err_inf_bound": None,  # filled by the caller with dt and h
        "beta_max": beta_max,
    }


def solve_and_store(pr, out, sample_seed, n_cells=4096, n_faces=(1365, 1365, 1366)):
    """Solve pr with the oracle to its FP64 floor and store the sampled record."""
    g = pr.grid
    t0 = time.time()
    res = oracle.projection_step(g, pr.C, pr.rho1, pr.rho2, pr.dt, pr.u, pr.v, pr.w, tol=1e-13)
    t1 = time.time()
    b0 = oracle.remove_mean(res.rhs)
    bound = oracle_error_bound(res, b0)
    bound["u_err_inf_bound"] = 2.0 * pr.dt * bound["beta_max"] * bound["p_err_inf_bound"] / g.h
    ustar_max = max(float(np.abs(a).max()) for a in (pr.u, pr.v, pr.w))
    bound["u_rel_err_bound"] = bound["u_err_inf_bound"] / ustar_max
    rng = np.random.default_rng(sample_seed)
    cells = rng.integers(0, g.ncells, size=n_cells)
    faces = [rng.integers(0, res.u[a].size, size=n_faces[a]) for a in range(3)]
    rec = {
        "workload": pr.name,
        "grid": [g.nx, g.ny, g.nz], "h": g.h, "bc": list(g.bc),
        "rho1": pr.rho1, "rho2": pr.rho2, "dt": pr.dt,
        "C_sha256": hashlib.sha256(np.ascontiguousarray(pr.C).tobytes()).hexdigest(),
        "oracle": {"cg_iters": res.cg.iters, "stagnated": res.cg.stagnated,
                   "rel_res_l2": res.cg.rel_res_l2, "rel_res_linf": res.cg.rel_res_linf,
                   "lanczos_lambda_min": bound["lanczos_lambda_min"],
                   "lanczos_lambda_max": bound["lanczos_lambda_max"],
                   "seconds": t1 - t0, "threads": int(os.environ.get("OMP_NUM_THREADS",
                                                                     os.cpu_count()))},
        "bound": bound,
        "ustar_max_abs": ustar_max,
        "p_max_abs": float(np.abs(res.p).max()),
        "cells": cells.tolist(),
        "p": res.p.ravel()[cells].tolist(),
        "faces": [f.tolist() for f in faces],
        "u": [res.u[a].ravel()[faces[a]].tolist() for a in range(3)],
        "u_max_abs": [float(np.abs(res.u[a]).max()) for a in range(3)],
    }
    with open(out, "w") as fh:
        json.dump(rec, fh)
    print(out, rec["oracle"], rec["bound"])


def main(n=256, out=None):
    out = out or os.path.join(os.path.dirname(os.path.abspath(__file__)), f"drops{n}_walls_z.json")
    solve_and_store(pi.config2(n=n), out, [300, n])


if __name__ == "__main__":
    main(int(sys.argv[1]) if len(sys.argv) > 1 else 256)
