"""Implicit viscous step on the staggered grid: plain FP64 CPU oracle.

TEST INFRASTRUCTURE ONLY: only the tests may import this module; the
library's product path never calls it.  Arithmetic in numpy and scipy.sparse
(FP64), written from the PARIS paper (arXiv 2012.11744), Sec. 3.2.3
("Implicitation of the viscous terms", Eq. muelliptic):

    u* - tau nu_f Lap_h u* = u^n        for each velocity component,

each component on its own face grid, Lap_h the 7-point Laplacian with
spacing h.  Readings (the paper prints the coefficient as mu; its predictor,
Eq. nonconspredictedvel, divides the viscous term by rho):

* the coefficient is the kinematic viscosity at the face, nu_f = mu_f / rho_f,
  with mu and rho from Eq. muH in the two cells sharing the face and both
  averaged arithmetically (the reading already used for rho in the
  projection), so nu_f = (mu_L + mu_R) / (rho_L + rho_R);
* periodic axes wrap;
* along a wall axis the normal component is zero on the wall faces, which
  are not unknowns;
* a tangential component next to a wall satisfies no-slip (Sec. 2.2: the
  fluid sticks to the wall, here at rest): the value beyond the wall is minus
  the first interior value (zero velocity on the wall, half a cell away).

Multiplying by 1/(tau nu_f) gives the symmetric positive definite form
(diag(1/(tau nu)) - Lap_h) u* = u^n / (tau nu), which is what `solve` uses.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

PERIODIC = 0
WALL = 1


def _n(grid):
    return (grid.nx, grid.ny, grid.nz)


def unknown_shape(grid, comp):
    """numpy shape (z, y, x) of the unknowns of component `comp` (0 = u, 1 = v,
    2 = w): the face grid without the wall faces of its own axis."""
    n = list(_n(grid))  # cells per axis (x, y, z)
    if grid.bc[comp] == WALL:
        n[comp] -= 1  # faces 1 .. n-1
    return (n[2], n[1], n[0])


def interior(grid, comp, face_array):
    """The unknowns (a view) of a full face array of component `comp`."""
    a = np.asarray(face_array)
    if grid.bc[comp] != WALL:
        return a
    sl = [slice(None)] * 3
    sl[2 - comp] = slice(1, -1)
    return a[tuple(sl)]


def embed(grid, comp, unknowns):
    """A full face array of component `comp` with the given interior values and
    zeros on its wall faces."""
    n = list(_n(grid))
    if grid.bc[comp] == WALL:
        n[comp] += 1
    out = np.zeros((n[2], n[1], n[0]))
    sl = [slice(None)] * 3
    if grid.bc[comp] == WALL:
        sl[2 - comp] = slice(1, -1)
    out[tuple(sl)] = unknowns
    return out


def face_nu(grid, comp, C, mu1, mu2, rho1, rho2):
    """nu_f = (mu_L + mu_R) / (rho_L + rho_R) on the unknowns of component `comp`,
    mu and rho from Eq. muH with the volume fraction C as the Heaviside function."""
    C = np.asarray(C, dtype=np.float64)
    mu = mu1 * C + mu2 * (1.0 - C)
    rho = rho1 * C + rho2 * (1.0 - C)
    ax = 2 - comp  # numpy axis of the component's direction
    n = C.shape[ax]
    if grid.bc[comp] == WALL:
        # interior face i (1 .. n-1) between cells i-1 and i
        lo = np.take(mu, np.arange(0, n - 1), axis=ax), np.take(rho, np.arange(0, n - 1), axis=ax)
        hi = np.take(mu, np.arange(1, n), axis=ax), np.take(rho, np.arange(1, n), axis=ax)
    else:
        # face i (0 .. n-1) between cells i-1 (wrapped) and i
        lo = np.roll(mu, 1, axis=ax), np.roll(rho, 1, axis=ax)
        hi = mu, rho
    return (lo[0] + hi[0]) / (lo[1] + hi[1])


def _second_difference(m, kind, h):
    """1-D second difference on m points, scaled by 1/h^2.
    kind: 'periodic' (wrap), 'dirichlet' (the neighbours beyond the ends are 0),
    'noslip' (the neighbour beyond each end is minus the end value)."""
    if kind == "periodic" and m == 1:
        return sp.csr_matrix((1, 1))  # the point is its own neighbour on both sides
    main = np.full(m, -2.0)
    off = np.ones(m - 1)
    if kind == "noslip":
        main[0] -= 1.0
        main[-1] -= 1.0
    T = sp.diags([off, main, off], [-1, 0, 1], shape=(m, m), format="lil")
    if kind == "periodic" and m > 1:
        T[0, m - 1] += 1.0
        T[m - 1, 0] += 1.0
    return (T.tocsr() / (h * h)).astype(np.float64)


def laplacian(grid, comp):
    """The 7-point Laplacian on the unknowns of component `comp` (CSR, unknowns
    flattened in (z, y, x) order)."""
    shape = unknown_shape(grid, comp)  # (z, y, x)
    mats = []
    for axis in range(3):  # x, y, z
        m = shape[2 - axis]
        if grid.bc[axis] == PERIODIC:
            kind = "periodic"
        elif axis == comp:
            kind = "dirichlet"
        else:
            kind = "noslip"
        mats.append(_second_difference(m, kind, grid.h))
    Ix, Iy, Iz = (sp.identity(shape[2 - a], format="csr") for a in range(3))
    # unknown (k, j, i) at index (k*ny + j)*nx + i: x fastest
    L = (sp.kron(Iz, sp.kron(Iy, mats[0])) + sp.kron(Iz, sp.kron(mats[1], Ix)) +
         sp.kron(mats[2], sp.kron(Iy, Ix)))
    return L.tocsr()


def spd_operator(grid, comp, nu, tau):
    """diag(1/(tau nu)) - Lap_h on the unknowns (symmetric positive definite)."""
    d = 1.0 / (tau * np.asarray(nu, dtype=np.float64).ravel())
    return (sp.diags(d) - laplacian(grid, comp)).tocsr()


def solve(grid, comp, nu, tau, un, tol=1e-13, max_iter=100000, stats=None):
    """u* of Eq. muelliptic for component `comp`: `un` and the result are arrays
    of the unknowns (unknown_shape).  tau = 0 returns u^n.  `stats` (a dict,
    optional) receives the number of CG iterations under "iters"."""
    un = np.asarray(un, dtype=np.float64)
    if tau == 0.0:
        if stats is not None:
            stats["iters"] = 0
        return un.copy()
    A = spd_operator(grid, comp, nu, tau)
    b = (un / (tau * np.asarray(nu, dtype=np.float64))).ravel()
    count = [0]

    def tick(_xk):
        count[0] += 1

    x, info = spla.cg(A, b, x0=un.ravel().copy(), rtol=tol, atol=0.0, maxiter=max_iter, callback=tick)
    if info != 0:
        raise RuntimeError(f"viscous CG did not converge (info {info})")
    if stats is not None:
        stats["iters"] = count[0]
    return x.reshape(un.shape)


def residual(grid, comp, nu, tau, us, un):
    """u* - tau nu Lap_h u* - u^n on the unknowns (the equation as printed)."""
    us = np.asarray(us, dtype=np.float64)
    lap = (laplacian(grid, comp) @ us.ravel()).reshape(us.shape)
    return us - tau * np.asarray(nu) * lap - np.asarray(un)
