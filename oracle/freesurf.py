"""Free-surface projections: plain FP64 CPU oracle (numpy and scipy.sparse).

TEST INFRASTRUCTURE ONLY: only the tests may import this module; the
library's product path never calls it.  Written from Sec. 3.7.5 of the PARIS
paper (arXiv 2012.11744), "Free-surface flow solver", with the boundary
condition of Sec. 2 "Free-surface flow" (Eq. free_surf_norm_bc):

* gfm_projection: the projection solved in the liquid only (the cells with
  C < 1/2, C the gas fraction as in that section), with the liquid density
  alone (beta = 1/rho_l on every face).  A face between a liquid cell and a
  gas cell takes the gradient of Eq. mod_branches, (p_s - p_c)/delta with
  delta = theta h the distance from the liquid node to the interface, and
  the interface pressure of Eq. Laplace_num, p_s = p_gas + sigma (kappa_c +
  kappa_g)/2 with p_gas the pressure of the gas cell (the polytropic value
  of Eq. polygas, given per cell).  The corrected velocity (Eq. fotm) uses
  the same gradients; gas-gas faces are left as they are (their values are
  extrapolated later); the gas cells report p_gas.
* gas_layers / phantom_projection: the "phantom" projection of "Ensuring
  volume conservation": a Poisson equation div grad P = div u (no density,
  no dt) in the first two layers of gas cells, a zero gradient on the faces
  to the liquid (their solved velocities kept), P = 0 in the gas cells
  beyond; only the faces between two gas cells at least one of which is in
  the two layers are corrected, u <- u - grad P.

Readings (where the paper leaves a choice):
* the layers are counted through faces: layer 1 the gas cells with a liquid
  face neighbour, layer 2 the other gas cells with a face neighbour in
  layer 1;
* theta (one value per face, used only on liquid-gas faces) is the distance
  along the face's axis from the liquid cell's node to the interface in
  units of h, in (0, 1];
* kappa enters Eq. Laplace_num with the sign the caller gives it;
* domain walls are closed faces (no flux, zero velocity) as in Sec. 3.8.

Both systems are assembled face by face with pure-Python loops (small grids
only) and solved with a direct sparse factorisation (scipy.sparse.linalg.
spsolve).  The assembled matrix is the negative of the discrete operator
(symmetric positive definite when every liquid region touches the gas, and
every two-layer region touches the gas beyond).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

PERIODIC = 0
WALL = 1


def _face_shape(grid, axis):
    n = [grid.nz, grid.ny, grid.nx]
    n[2 - axis] += 1 if grid.bc[axis] == WALL else 0
    return tuple(n)


def _faces(grid, axis):
    """Every face of an axis as (face index tuple, lower cell, upper cell);
    a wall face has None on its outer side."""
    n = (grid.nx, grid.ny, grid.nz)[axis]
    wall = grid.bc[axis] == WALL
    for k in range(grid.nz):
        for j in range(grid.ny):
            for i in range(grid.nx):
                cell = [k, j, i]
                # the lower face of this cell: between cell - e_axis (wrapped) and cell
                f = (k, j, i)
                lo = list(cell)
                lo[2 - axis] -= 1
                if lo[2 - axis] < 0:
                    lo = None if wall else [*lo[:2 - axis], n - 1, *lo[3 - axis:]]
                yield f, (tuple(lo) if lo is not None else None), tuple(cell)
    if wall:  # the upper wall faces
        if axis == 0:
            for k in range(grid.nz):
                for j in range(grid.ny):
                    yield (k, j, n), (k, j, n - 1), None
        elif axis == 1:
            for k in range(grid.nz):
                for i in range(grid.nx):
                    yield (k, n, i), (k, n - 1, i), None
        else:
            for j in range(grid.ny):
                for i in range(grid.nx):
                    yield (n, j, i), (n - 1, j, i), None


def _divergence(grid, u, v, w):
    """(1/h) sum over the axes of (u_{+face} - u_{-face}) at every cell."""
    d = np.zeros((grid.nz, grid.ny, grid.nx))
    for axis, a in enumerate((u, v, w)):
        for f, lo, hi in _faces(grid, axis):
            if lo is not None:
                d[lo] += a[f]
            if hi is not None:
                d[hi] -= a[f]
    return d / grid.h


def liquid_mask(C):
    """Sec. 3.7.5: only the cells with C < 1/2 are solved (C = 0 in the liquid)."""
    return np.asarray(C) < 0.5


def interface_pressure(p_gas, kappa, sigma, c_liq, c_gas):
    """Eq. Laplace_num: p_s = p_gas (of the gas cell) + sigma (kappa_c + kappa_g)/2."""
    return p_gas[c_gas] + sigma * 0.5 * (kappa[c_liq] + kappa[c_gas])


def gfm_projection(grid, C, rho_l, dt, u, v, w, p_gas, theta=None, kappa=None, sigma=0.0):
    """The free-surface projection of Sec. 3.7.5.  Returns (p, (u, v, w), A, b):
    p in the liquid from the solve and p_gas in the gas, the corrected
    velocity, and the assembled SPD system A p_liq = b."""
    liq = liquid_mask(C)
    p_gas = np.asarray(p_gas, dtype=np.float64)
    kappa = np.zeros(liq.shape) if kappa is None else np.asarray(kappa, dtype=np.float64)
    theta = [np.ones(_face_shape(grid, a)) for a in range(3)] if theta is None else \
        [np.asarray(t, dtype=np.float64) for t in theta]
    beta = 1.0 / rho_l
    h2 = grid.h * grid.h
    us = [np.array(a, dtype=np.float64) for a in (u, v, w)]
    # the solved velocities on the walls are zero
    for axis in range(3):
        for f, lo, hi in _faces(grid, axis):
            if lo is None or hi is None:
                us[axis][f] = 0.0
    idx = -np.ones(liq.shape, np.int64)
    cells = list(zip(*np.nonzero(liq)))
    for n, c in enumerate(cells):
        idx[c] = n
    div = _divergence(grid, *us)
    b = np.array([-div[c] / dt for c in cells])
    rows, cols, vals = [], [], []
    diag = np.zeros(len(cells))
    # every face joining a liquid cell to another cell: a flux term in each
    # liquid cell it touches (Eq. poisson with the gradients of Eq. mod_branches)
    for axis in range(3):
        for f, lo, hi in _faces(grid, axis):
            if lo is None or hi is None:
                continue
            ll, lh = bool(liq[lo]), bool(liq[hi])
            if ll and lh:
                cf = beta / h2
                for c, o in ((lo, hi), (hi, lo)):
                    diag[idx[c]] += cf
                    rows.append(idx[c])
                    cols.append(idx[o])
                    vals.append(-cf)
            elif ll or lh:
                c, gcell = (lo, hi) if ll else (hi, lo)
                cf = beta / (theta[axis][f] * h2)
                diag[idx[c]] += cf
                b[idx[c]] += cf * interface_pressure(p_gas, kappa, sigma, c, gcell)
    rows += list(range(len(cells)))
    cols += list(range(len(cells)))
    vals += list(diag)
    A = sp.csr_matrix((vals, (rows, cols)), shape=(len(cells), len(cells)))
    x = spla.spsolve(A.tocsc(), b)
    p = p_gas.copy()
    for n, c in enumerate(cells):
        p[c] = x[n]
    # Eq. fotm with the same face gradients; gas-gas and wall faces untouched
    for axis in range(3):
        for f, lo, hi in _faces(grid, axis):
            if lo is None or hi is None:
                continue
            ll, lh = bool(liq[lo]), bool(liq[hi])
            if ll and lh:
                g = (p[hi] - p[lo]) / grid.h
            elif ll:
                g = (interface_pressure(p_gas, kappa, sigma, lo, hi) - p[lo]) / (theta[axis][f] * grid.h)
            elif lh:
                g = (p[hi] - interface_pressure(p_gas, kappa, sigma, hi, lo)) / (theta[axis][f] * grid.h)
            else:
                continue
            us[axis][f] -= dt * beta * g
    return p, tuple(us), A, b


def gas_layers(grid, C):
    """Cell classes of the phantom projection: 0 liquid, 1 the first two
    layers of gas cells (through faces), 2 the gas beyond."""
    liq = liquid_mask(C)
    cls = np.full(liq.shape, 2, np.int8)
    cls[liq] = 0

    def touches(mask):
        t = np.zeros(mask.shape, bool)
        for axis in range(3):
            for f, lo, hi in _faces(grid, axis):
                if lo is None or hi is None:
                    continue
                if mask[lo]:
                    t[hi] = True
                if mask[hi]:
                    t[lo] = True
        return t

    l1 = touches(liq) & ~liq
    l2 = touches(l1) & ~liq & ~l1
    cls[l1 | l2] = 1
    return cls


def phantom_projection(grid, C, u, v, w):
    """The phantom projection of "Ensuring volume conservation".  Returns
    (P, (u, v, w), cls): P on the two gas layers (0 elsewhere), the velocity
    with the extrapolated faces corrected, and the cell classes."""
    cls = gas_layers(grid, C)
    h2 = grid.h * grid.h
    us = [np.array(a, dtype=np.float64) for a in (u, v, w)]
    cells = list(zip(*np.nonzero(cls == 1)))
    idx = -np.ones(cls.shape, np.int64)
    for n, c in enumerate(cells):
        idx[c] = n
    div = _divergence(grid, *us)
    b = np.array([-div[c] for c in cells])
    rows, cols, vals = [], [], []
    diag = np.zeros(len(cells))
    for axis in range(3):
        for f, lo, hi in _faces(grid, axis):
            if lo is None or hi is None or cls[lo] == 0 or cls[hi] == 0:
                continue  # walls and the faces to the liquid: no gradient term
            for c, o in ((lo, hi), (hi, lo)):
                if cls[c] != 1:
                    continue
                diag[idx[c]] += 1.0 / h2
                if cls[o] == 1:
                    rows.append(idx[c])
                    cols.append(idx[o])
                    vals.append(-1.0 / h2)
    rows += list(range(len(cells)))
    cols += list(range(len(cells)))
    vals += list(diag)
    A = sp.csr_matrix((vals, (rows, cols)), shape=(len(cells), len(cells)))
    x = spla.spsolve(A.tocsc(), b) if cells else np.zeros(0)
    P = np.zeros(cls.shape)
    for n, c in enumerate(cells):
        P[c] = x[n]
    for axis in range(3):
        for f, lo, hi in _faces(grid, axis):
            if lo is None or hi is None or cls[lo] == 0 or cls[hi] == 0:
                continue
            if cls[lo] == 1 or cls[hi] == 1:
                us[axis][f] -= (P[hi] - P[lo]) / grid.h
    return P, tuple(us), cls
