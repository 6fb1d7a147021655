"""Write tests/golden/viscous256_drops.json from full FP64 CPU-oracle solves of
the implicit viscous step (Eq. muelliptic) on the 256^3 drop field (periodic
x, y; walls z; rho 1000/1), one per velocity component.

Calls only the oracle and the seeded input generator.  Viscosities mu 1e-3
(fluid 1) and 1.8e-5 (fluid 2), nu_f from Eq. muH means, tau = 4 h^2 / max
nu_f over the three components, u^n = the workload's u*.  Stored: a checksum
of the volume fraction, tau, and per component the oracle's CG iteration
count, its relative residual of the SPD form, max |u*| and u* at 2048 seeded
unknowns (indices into the component's unknowns, x fastest).
Run:  python tests/golden/make_viscous256_golden.py  (a few minutes).
"""
import hashlib
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)
import paris_inputs as pi  # noqa: E402
from oracle import viscous as V  # noqa: E402

MU1, MU2 = 1.0e-3, 1.8e-5
TAU_NU_OVER_H2 = 4.0


def main(n=256, out=None):
    out = out or os.path.join(os.path.dirname(os.path.abspath(__file__)), f"viscous{n}_drops.json")
    pr = pi.config2(n=n)
    g = pr.grid
    nus = [V.face_nu(g, c, pr.C, MU1, MU2, pr.rho1, pr.rho2) for c in range(3)]
    tau = TAU_NU_OVER_H2 * g.h ** 2 / max(float(nu.max()) for nu in nus)
    rng = np.random.default_rng([400, n])
    comps = []
    for c in range(3):
        un = V.interior(g, c, (pr.u, pr.v, pr.w)[c])
        info = {}
        t0 = time.time()
        x = V.solve(g, c, nus[c], tau, un, tol=1e-13, stats=info)
        t1 = time.time()
        A = V.spd_operator(g, c, nus[c], tau)
        b = (un / (tau * nus[c])).ravel()
        r = b - A @ x.ravel()
        idx = rng.integers(0, x.size, size=2048)
        comps.append({"iters": info["iters"], "seconds": t1 - t0,
                      "rel_res_l2": float(np.linalg.norm(r) / np.linalg.norm(b)),
                      "rel_res_linf": float(np.abs(r).max() / np.abs(b).max()),
                      "x_max_abs": float(np.abs(x).max()),
                      "unknowns": idx.tolist(), "x": x.ravel()[idx].tolist()})
        print(c, info["iters"], comps[-1]["rel_res_l2"], f"{t1 - t0:.1f} s", flush=True)
    rec = {"workload": f"drops{n}_walls_z", "grid": [g.nx, g.ny, g.nz], "h": g.h, "bc": list(g.bc),
           "rho1": pr.rho1, "rho2": pr.rho2, "mu1": MU1, "mu2": MU2,
           "tau_nu_over_h2": TAU_NU_OVER_H2, "tau": tau,
           "C_sha256": hashlib.sha256(np.ascontiguousarray(pr.C).tobytes()).hexdigest(),
           "threads": os.cpu_count(), "components": comps}
    with open(out, "w") as fh:
        json.dump(rec, fh)
    print(out)


if __name__ == "__main__":
    main(int(sys.argv[1]) if len(sys.argv) > 1 else 256)
