"""Write tests/golden/drops256_walls_z.json from a full FP64 CPU-oracle solve of
the 256^3 drop field (periodic x, y; walls z; rho 1000/1; dt = 1e-4).

Calls only the oracle and the seeded input generator.  Stored: a checksum of
the volume fraction (so a test can confirm it regenerates the same input), the
oracle's CG iteration count and residuals, its Lanczos eigenvalue estimates,
and p and the corrected velocity at 4096 seeded sample points.
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


def main(n=256, out=None):
    out = out or os.path.join(os.path.dirname(os.path.abspath(__file__)), f"drops{n}_walls_z.json")
    pr = pi.config2(n=n)
    g = pr.grid
    t0 = time.time()
    res = oracle.projection_step(g, pr.C, pr.rho1, pr.rho2, pr.dt, pr.u, pr.v, pr.w, tol=1e-13)
    t1 = time.time()
    lmin, lmax = res.cg.lanczos_extremes()
    rng = np.random.default_rng([300, n])
    cells = rng.integers(0, g.ncells, size=4096)
    faces = [rng.integers(0, res.u[a].size, size=1365) for a in range(3)]
    rec = {
        "workload": f"drops{n}_walls_z",
        "grid": [g.nx, g.ny, g.nz], "h": g.h, "bc": list(g.bc),
        "rho1": pr.rho1, "rho2": pr.rho2, "dt": pr.dt,
        "C_sha256": hashlib.sha256(np.ascontiguousarray(pr.C).tobytes()).hexdigest(),
        "oracle": {"cg_iters": res.cg.iters, "stagnated": res.cg.stagnated,
                   "rel_res_l2": res.cg.rel_res_l2, "rel_res_linf": res.cg.rel_res_linf,
                   "lanczos_lambda_min": lmin, "lanczos_lambda_max": lmax,
                   "seconds": t1 - t0, "threads": os.cpu_count()},
        "p_max_abs": float(np.abs(res.p).max()),
        "cells": cells.tolist(),
        "p": res.p.ravel()[cells].tolist(),
        "faces": [f.tolist() for f in faces],
        "u": [res.u[a].ravel()[faces[a]].tolist() for a in range(3)],
        "u_max_abs": [float(np.abs(res.u[a]).max()) for a in range(3)],
    }
    with open(out, "w") as fh:
        json.dump(rec, fh)
    print(out, rec["oracle"])


if __name__ == "__main__":
    main(int(sys.argv[1]) if len(sys.argv) > 1 else 256)
