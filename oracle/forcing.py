"""Capillary and gravity forcing of the predictor on the faces: plain FP64 CPU oracle.

TEST INFRASTRUCTURE ONLY: only the tests may import this module; the
library's product path never calls it.  numpy, FP64, written from the PARIS
paper (arXiv 2012.11744):

* the non-conservative predictor, Eq. nonconspredictedvel, adds
  tau (L_cap + L_ext) / rho^{n+1} to u^n (its advection and viscous terms are
  left out here: the viscous one is the implicit step of Eq. muelliptic);
* the capillary term in CSF form, Eq. csf2: -sigma kappa^h grad^h C;
* gravity as the external force, L_ext = rho g (Sec. 2).

On every face f that is not a wall face, between cells L and R along the
face's axis a:

    a_f = -sigma kappa_f (C_R - C_L) / (h rho_f) + g_a,     u*_f = u^n_f + tau a_f,

and a_f = 0, u*_f = 0 on wall faces.  Readings:

* rho_f = (rho_L + rho_R)/2 with rho = rho1 C + rho2 (1 - C) (Eq. muH), the face
  density of the projection, so that with a constant kappa the capillary
  acceleration is beta_f times the face gradient of -sigma kappa C: a discrete
  gradient with the projection's own weights (the well-balanced property the
  paper claims for CSF);
* kappa_f = (kappa_L + kappa_R)/2: the paper does not say how the cell
  curvature reaches the faces;
* L_ext / rho at a face is rho_f g / rho_f = g exactly;
* the sign of kappa is the one that makes Eq. csf2 and the jump condition
  Eq. jump1 agree: with n the unit normal pointing out of fluid 1
  (n delta_S = -grad H), a sphere of fluid 1 of radius R has kappa = -2/R, and
  the pressure inside exceeds the outside by 2 sigma / R.

Face arrays use the library's layout: face i of axis a lies between cells
i-1 (wrapped along a periodic axis) and i; along a wall axis the array has
n+1 faces and faces 0 and n are the walls.  Arrays are numpy (z, y, x).
"""
from __future__ import annotations

import numpy as np

PERIODIC = 0
WALL = 1


def face_shape(grid, axis):
    n = [grid.nz, grid.ny, grid.nx]
    n[2 - axis] += 1 if grid.bc[axis] == WALL else 0
    return tuple(n)


def _neighbours(grid, q, axis):
    """(q_L, q_R) of the cell field q on every face of `axis` that is not a
    wall face, and the slice of the face array those faces occupy."""
    ax = 2 - axis  # numpy axis
    n = q.shape[ax]
    sl = [slice(None)] * 3
    if grid.bc[axis] == WALL:
        lo = np.take(q, np.arange(0, n - 1), axis=ax)
        hi = np.take(q, np.arange(1, n), axis=ax)
        sl[ax] = slice(1, n)
    else:
        lo = np.roll(q, 1, axis=ax)
        hi = q
    return lo, hi, tuple(sl)


def face_acceleration(grid, C, kappa, sigma, gravity, rho1, rho2):
    """(a_x, a_y, a_z): the capillary (Eq. csf2) plus gravity acceleration on
    the faces, 0 on wall faces.  C, kappa: cell arrays; gravity: (g_x, g_y, g_z)."""
    C = np.asarray(C, dtype=np.float64)
    kappa = np.broadcast_to(np.asarray(kappa, dtype=np.float64), C.shape)
    rho = rho1 * C + rho2 * (1.0 - C)
    out = []
    for axis in range(3):
        a = np.zeros(face_shape(grid, axis))
        cl, cr, sl = _neighbours(grid, C, axis)
        kl, kr, _ = _neighbours(grid, kappa, axis)
        rl, rr, _ = _neighbours(grid, rho, axis)
        rho_f = (rl + rr) / 2.0
        kappa_f = (kl + kr) / 2.0
        a[sl] = -sigma * kappa_f * (cr - cl) / (grid.h * rho_f) + gravity[axis]
        out.append(a)
    return tuple(out)


def predictor(grid, u, v, w, C, kappa, sigma, gravity, rho1, rho2, tau):
    """u* = u^n + tau a_f on the faces (the capillary and gravity part of
    Eq. nonconspredictedvel); wall faces 0."""
    acc = face_acceleration(grid, C, kappa, sigma, gravity, rho1, rho2)
    out = []
    for axis, (un, a) in enumerate(zip((u, v, w), acc)):
        us = np.asarray(un, dtype=np.float64) + tau * a
        if grid.bc[axis] == WALL:
            sl = [slice(None)] * 3
            for end in (0, -1):
                sl[2 - axis] = end
                us[tuple(sl)] = 0.0
        out.append(us)
    return tuple(out)
