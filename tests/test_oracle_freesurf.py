"""Pins of the free-surface oracle (oracle/freesurf.py, Sec. 3.7.5 "Free-
surface flow solver" and "Ensuring volume conservation") against what the
paper and the mathematics fix, on the CPU.

Each test names the mistake it would catch: theta taken from the wrong side
or as 1 - theta, the interface pressure of Eq. Laplace_num with a wrong sign
or one-sided curvature, a gradient of Eq. mod_branches that disagrees with
the system, layers counted wrongly, a phantom correction that touches the
solved velocities."""
import numpy as np
import pytest

import oracle
import paris_inputs as pi
from oracle import freesurf as FS

P, W = pi.PERIODIC, pi.WALL


def slab(grid, k_lo, k_hi):
    """Gas fraction 1 outside planes k_lo..k_hi, 0 inside (a liquid slab)."""
    C = np.ones(grid.shape)
    C[k_lo:k_hi + 1] = 0.0
    return C


@pytest.mark.parametrize("bc_z", [P, W], ids=["z_periodic", "z_walls"])
def test_linear_profile_between_two_free_surfaces(bc_z):
    """A liquid slab (planes 2..7 of 10) with the interfaces theta_lo h below
    plane 2 and theta_hi h above plane 7, gas pressures P_lo and P_hi, two
    curvatures (liquid, gas) and u* = 0: the exact solution is linear in z
    through the two interface pressures, and every discrete equation (interior
    second differences and the cut faces of Eq. mod_branches) holds exactly
    for it.  A theta taken as 1 - theta, from the other side, or a p_s
    without the mean curvature of Eq. Laplace_num all move p."""
    g = pi.Grid(4, 3, 10, 0.1, (P, P, bc_z))
    k_lo, k_hi = 2, 7
    C = slab(g, k_lo, k_hi)
    th_lo, th_hi = 0.23, 0.71
    theta = [np.ones(g.face_shape(a)) for a in range(3)]
    theta[2][k_lo] = th_lo       # face between planes 1 and 2
    theta[2][k_hi + 1] = th_hi   # face between planes 7 and 8
    P_lo, P_hi, sigma = 3.0, -1.5, 0.07
    p_gas = np.where(np.arange(g.nz)[:, None, None] < k_lo, P_lo, P_hi) * np.ones(g.shape)
    kappa = np.where(C < 0.5, 12.0, -4.0)
    zero = [np.zeros(g.face_shape(a)) for a in range(3)]
    p, u, A, b = FS.gfm_projection(g, C, 800.0, 1e-3, *zero, p_gas, theta, kappa, sigma)
    ps_lo = P_lo + sigma * 0.5 * (12.0 - 4.0)
    ps_hi = P_hi + sigma * 0.5 * (12.0 - 4.0)
    z = (np.arange(g.nz) + 0.5) * g.h
    z_lo, z_hi = z[k_lo] - th_lo * g.h, z[k_hi] + th_hi * g.h
    slope = (ps_hi - ps_lo) / (z_hi - z_lo)
    want = ps_lo + slope * (z - z_lo)
    for k in range(k_lo, k_hi + 1):
        np.testing.assert_allclose(p[k], want[k], rtol=1e-12, atol=1e-12)
    np.testing.assert_array_equal(p[:k_lo], P_lo)
    np.testing.assert_array_equal(p[k_hi + 1:], P_hi)
    # u = -dt beta slope on every z face touching the liquid, 0 in x and y
    for k in range(k_lo, k_hi + 2):
        np.testing.assert_allclose(u[2][k], -1e-3 / 800.0 * slope, rtol=1e-11)
    assert max(np.abs(u[0]).max(), np.abs(u[1]).max()) <= 1e-12 * abs(1e-3 / 800.0 * slope)


def test_constant_curvature_gives_the_laplace_pressure():
    """Gas bubbles in liquid, one gas pressure P0 and a constant curvature:
    p = P0 + sigma kappa in every liquid cell and u* = 0 stays 0, for any
    theta (the constant solves every equation)."""
    g = pi.Grid(12, 10, 8, 1 / 12, (P, W, P))
    rng = np.random.default_rng(5)
    C = (rng.random(g.shape) < 0.3).astype(float)
    theta = [rng.uniform(0.05, 1.0, g.face_shape(a)) for a in range(3)]
    zero = [np.zeros(g.face_shape(a)) for a in range(3)]
    p, u, A, b = FS.gfm_projection(g, C, 1000.0, 1e-3, *zero, np.full(g.shape, 2.5), theta,
                                   np.full(g.shape, -30.0), 0.07)
    liq = C < 0.5
    np.testing.assert_allclose(p[liq], 2.5 + 0.07 * -30.0, rtol=1e-12)
    assert np.all(p[~liq] == 2.5)
    for a in range(3):
        assert np.abs(u[a]).max() <= 1e-12


@pytest.mark.parametrize("grid", [pi.Grid(10, 9, 8, 0.1, (P, P, P)), pi.Grid(9, 8, 11, 0.1, (W, P, W))],
                         ids=["ppp", "wpw"])
def test_gradient_field_is_removed(grid):
    """u* = dt beta grad phi with the gradients of Eq. mod_branches (written
    out here face by face from the paper): the projection returns p = phi in
    the liquid and u = 0 on every face touching the liquid, and leaves the
    gas-gas faces as they were."""
    rng = np.random.default_rng(11)
    C = (rng.random(grid.shape) < 0.35).astype(float)
    liq = C < 0.5
    theta = [rng.uniform(0.1, 1.0, grid.face_shape(a)) for a in range(3)]
    kappa = rng.normal(size=grid.shape)
    p_gas = rng.normal(size=grid.shape)
    sigma, rho_l, dt = 0.3, 50.0, 2e-3
    phi = rng.normal(size=grid.shape)
    us = [rng.normal(size=grid.face_shape(a)) for a in range(3)]  # gas-gas faces keep these
    n = (grid.nx, grid.ny, grid.nz)
    for a in range(3):
        ax = 2 - a
        for idx in np.ndindex(grid.face_shape(a)):
            m = idx[ax]
            wall = grid.bc[a] == W
            if wall and (m == 0 or m == n[a]):
                us[a][idx] = 0.0
                continue
            hi = list(idx)
            hi[ax] = m % n[a]
            lo = list(idx)
            lo[ax] = (m - 1) % n[a]
            hi, lo = tuple(hi), tuple(lo)
            if liq[lo] and liq[hi]:
                gr = (phi[hi] - phi[lo]) / grid.h
            elif liq[lo]:
                ps = p_gas[hi] + sigma * (kappa[lo] + kappa[hi]) / 2
                gr = (ps - phi[lo]) / (theta[a][idx] * grid.h)
            elif liq[hi]:
                ps = p_gas[lo] + sigma * (kappa[hi] + kappa[lo]) / 2
                gr = (phi[hi] - ps) / (theta[a][idx] * grid.h)
            else:
                continue
            us[a][idx] = dt / rho_l * gr
    p, u, A, b = FS.gfm_projection(grid, C, rho_l, dt, *us, p_gas, theta, kappa, sigma)
    np.testing.assert_allclose(p[liq], phi[liq], rtol=0, atol=1e-10 * np.abs(phi).max())
    np.testing.assert_array_equal(p[~liq], p_gas[~liq])
    umax = max(np.abs(x).max() for x in us)
    for a in range(3):
        touched = np.zeros(grid.face_shape(a), bool)
        ax = 2 - a
        for idx in np.ndindex(grid.face_shape(a)):
            m = idx[ax]
            if grid.bc[a] == W and (m == 0 or m == n[a]):
                continue
            hi = list(idx); hi[ax] = m % n[a]
            lo = list(idx); lo[ax] = (m - 1) % n[a]
            touched[idx] = liq[tuple(lo)] or liq[tuple(hi)]
        assert np.abs(u[a][touched]).max() <= 1e-10 * umax
        np.testing.assert_array_equal(u[a][~touched], us[a][~touched])


def test_system_is_spd_and_divergence_vanishes():
    """The assembled matrix is symmetric positive definite, and after the
    projection of a random u* the discrete divergence vanishes in every
    liquid cell (the C oracle's divergence, walls closed)."""
    g = pi.Grid(8, 7, 6, 0.125, (P, W, P))
    rng = np.random.default_rng(13)
    C = (rng.random(g.shape) < 0.4).astype(float)
    theta = [rng.uniform(0.2, 1.0, g.face_shape(a)) for a in range(3)]
    us = [rng.normal(size=g.face_shape(a)) for a in range(3)]
    p, u, A, b = FS.gfm_projection(g, C, 10.0, 0.01, *us, rng.normal(size=g.shape), theta,
                                   rng.normal(size=g.shape), 0.1)
    Ad = A.toarray()
    assert np.abs(Ad - Ad.T).max() == 0.0
    assert np.linalg.eigvalsh(Ad).min() > 0.0
    d = oracle.divergence(g, *u, dt=1.0)
    liq = C < 0.5
    assert np.abs(d[liq]).max() <= 1e-10 * max(np.abs(x).max() for x in us) / g.h


def test_gas_layers_of_a_single_liquid_cell():
    """One liquid cell in a periodic 9^3 box: layer 1 is its 6 face
    neighbours, layer 2 the 18 cells at face distance 2 (6 along the axes,
    12 across two axes), everything else is gas beyond."""
    g = pi.Grid(9, 9, 9, 1 / 9)
    C = np.ones(g.shape)
    C[4, 4, 4] = 0.0
    cls = FS.gas_layers(g, C)
    assert cls[4, 4, 4] == 0
    k, j, i = np.indices(g.shape)
    dist = np.abs(k - 4) + np.abs(j - 4) + np.abs(i - 4)
    np.testing.assert_array_equal(cls == 1, (dist >= 1) & (dist <= 2))
    assert np.count_nonzero(cls == 1) == 24


def test_phantom_projection_recovers_a_gradient():
    """u = grad phi on the faces among gas cells (phi = 0 beyond the two
    layers) and 0 on the faces to the liquid: P = phi on the two layers and
    every corrected face becomes 0; the faces beyond are left alone."""
    g = pi.Grid(12, 11, 10, 0.1, (P, P, W))
    rng = np.random.default_rng(17)
    C = np.ones(g.shape)
    C[3:8, 2:9, 2:7] = 0.0  # a liquid block
    cls = FS.gas_layers(g, C)
    phi = np.where(cls == 1, rng.normal(size=g.shape), 0.0)
    us = [rng.normal(size=g.face_shape(a)) for a in range(3)]
    n = (g.nx, g.ny, g.nz)
    corrected = []
    for a in range(3):
        ax = 2 - a
        mask = np.zeros(g.face_shape(a), bool)
        for idx in np.ndindex(g.face_shape(a)):
            m = idx[ax]
            if g.bc[a] == W and (m == 0 or m == n[a]):
                us[a][idx] = 0.0
                continue
            hi = list(idx); hi[ax] = m % n[a]; hi = tuple(hi)
            lo = list(idx); lo[ax] = (m - 1) % n[a]; lo = tuple(lo)
            if cls[lo] == 0 or cls[hi] == 0:
                if cls[lo] == 1 or cls[hi] == 1:
                    us[a][idx] = 0.0  # the solved velocity on a liquid face of the layers
                continue
            if cls[lo] == 1 or cls[hi] == 1:
                us[a][idx] = (phi[hi] - phi[lo]) / g.h
                mask[idx] = True
        corrected.append(mask)
    Pp, u, cls2 = FS.phantom_projection(g, C, *us)
    np.testing.assert_array_equal(cls2, cls)
    np.testing.assert_allclose(Pp, phi, rtol=0, atol=1e-11 * np.abs(phi).max())
    for a in range(3):
        assert np.abs(u[a][corrected[a]]).max() <= 1e-10
        np.testing.assert_array_equal(u[a][~corrected[a]], us[a][~corrected[a]])


def test_phantom_projection_makes_the_layers_divergence_free():
    """A random extrapolated field around gas bubbles in liquid (the gas
    reaching beyond two layers): after the projection the divergence is 0 in
    every layer cell, the faces touching the liquid are unchanged, and an
    already projected field is a fixed point (P = 0)."""
    g = pi.Grid(14, 12, 13, 1 / 14, (P, P, P))
    rng = np.random.default_rng(19)
    C = np.zeros(g.shape)
    C[2:10, 3:11, 1:12] = 1.0  # a gas pocket wider than four cells
    us = [rng.normal(size=g.face_shape(a)) for a in range(3)]
    Pp, u, cls = FS.phantom_projection(g, C, *us)
    d = oracle.divergence(g, *u, dt=1.0)
    assert np.abs(d[cls == 1]).max() <= 1e-10 * max(np.abs(x).max() for x in us) / g.h
    P2, u2, _ = FS.phantom_projection(g, C, *u)
    assert np.abs(P2).max() <= 1e-10 * np.abs(Pp).max()
    for a in range(3):
        np.testing.assert_allclose(u2[a], u[a], rtol=0, atol=1e-10)
