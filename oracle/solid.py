"""Solid cells in the projection: plain FP64 CPU oracle (numpy on top of the
C oracle).

TEST INFRASTRUCTURE ONLY: only the tests may import this module; the
library's product path never calls it.  Written from Sec. 3.8 of the PARIS
paper (arXiv 2012.11744), "Solid boundaries":

* a cell flag s = 1 outside the solid and 0 inside ("Lego" solids);
* link flags on the faces, used to block the velocity (u_f <- s_f u_f every
  time the velocity is updated) and to zero the pressure coefficients on the
  links (a Neumann condition for p on the solid's boundary), with A7 the sum
  of the remaining six coefficients.

Reading (the printed initialisation loop sets the flag of face i+1/2 from
the cell on one side only, while the text asks that the velocity and the
pressure correction be blocked on the solid region AND its boundary): a face
is open only when both cells it joins are fluid, s_f = s_L s_R, and wall
faces are closed as in Sec. 3.8's walls.  The solid cells then have no open
face: their pressure is not determined by the system, and is reported as 0.
The gauge is the mean over the fluid cells (a connected fluid region; a
region cut into parts would leave one free constant per part).
"""
from __future__ import annotations

import numpy as np

from . import divergence, face_coeffs, null_project, Operator, cg, project

PERIODIC = 0
WALL = 1


def face_flags(grid, fluid):
    """(s_x, s_y, s_z): 1 on every face whose two cells are fluid, 0 on faces
    touching a solid cell and on wall faces.  Face arrays in the library's
    layout (face i of an axis between cells i-1, wrapped, and i)."""
    s = np.asarray(fluid, dtype=np.float64)
    out = []
    for axis in range(3):
        ax = 2 - axis
        n = s.shape[ax]
        shape = list(s.shape)
        if grid.bc[axis] == WALL:
            shape[ax] = n + 1
            f = np.zeros(shape)
            lo = np.take(s, np.arange(0, n - 1), axis=ax)
            hi = np.take(s, np.arange(1, n), axis=ax)
            sl = [slice(None)] * 3
            sl[ax] = slice(1, n)
            f[tuple(sl)] = lo * hi
        else:
            f = np.roll(s, 1, axis=ax) * s
        out.append(f)
    return tuple(out)


def face_coeffs_solid(grid, C, rho1, rho2, fluid):
    """beta_f of Eq. muH (face_coeffs) times the link flag: 0 on the solid's
    boundary and on walls."""
    beta = face_coeffs(grid, C, rho1, rho2)
    flags = face_flags(grid, fluid)
    return tuple(b * f for b, f in zip(beta, flags))


def projection_step_solid(grid, C, rho1, rho2, dt, u, v, w, fluid, tol=1e-13, max_iter=200000):
    """The projection with solid cells: u* blocked (u*_f <- s_f u*_f),
    b = D u*/dt, b's null-space part removed (fluid mean, 0 in the solid),
    the masked system solved to tol by CG, p with its fluid mean removed and
    0 in the solid, then u = u* - dt beta_f (G p)_f blocked again.
    Returns (p, (u, v, w), beta, CGResult, rhs)."""
    flags = face_flags(grid, fluid)
    beta = face_coeffs_solid(grid, C, rho1, rho2, fluid)
    us = [np.asarray(a, dtype=np.float64) * f for a, f in zip((u, v, w), flags)]
    b = divergence(grid, *us, dt)
    b0 = null_project(b, fluid)
    op = Operator(grid, *beta)
    res = cg(op, -b0, tol=tol, max_iter=max_iter, fluid=fluid)
    p = null_project(res.x, fluid)
    uu = project(grid, *beta, p, dt, *us)
    uu = tuple(a * f for a, f in zip(uu, flags))
    op.close()
    return p, uu, beta, res, b
