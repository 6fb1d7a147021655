"""Pins of the predictor-forcing oracle (oracle/forcing.py: the capillary CSF
term of Eq. csf2 and gravity, as they enter Eq. nonconspredictedvel) against
hand-computed values and the projection's exact balances (CPU)."""
import numpy as np
import pytest

import oracle
import paris_inputs as pi
from oracle import forcing as F

P, W = pi.PERIODIC, pi.WALL


def test_hand_computed_face_values():
    """2x2x2 cells, h = 1/2, periodic x and y, walls in z; sigma 1/2, rho 3/1,
    g = (0.1, 0.2, -0.3).  C = 1/4 in cell (z0,y0,x0), 3/4 in (z0,y0,x1), else 0;
    kappa = 4 in (z0,y0,x1), else 2.  By hand:
      x-face 1 of row (z0,y0): rho_f = (1.5+2.5)/2 = 2, kappa_f = 3, dC/h = 1:
        -0.5*3*1/2 + 0.1 = -0.65
      x-face 0 of row (z0,y0) (across the periodic seam, L = cell x1):
        dC/h = -1: 0.75 + 0.1 = 0.85
      x-face 1 of row (z1,y0): no C jump: 0.1
      y-face 0 of column (z0,x0) (L = cell y1 by wrap): rho_f = 1.25, dC/h = 0.5,
        kappa_f = 2: -0.5*2*0.5/1.25 + 0.2 = -0.2;  y-face 1 there: 0.6
      z-face 1 at (y0,x0): rho_f = 1.25, dC/h = -0.5: 0.4 - 0.3 = 0.1
      z-face 1 at (y0,x1): rho_f = 1.75, kappa_f = 3, dC/h = -1.5: 9/7 - 0.3
      z-faces 0 and 2 are walls: 0."""
    grid = pi.Grid(2, 2, 2, 0.5, (P, P, W))
    C = np.zeros((2, 2, 2))
    C[0, 0, 0], C[0, 0, 1] = 0.25, 0.75
    kappa = np.full((2, 2, 2), 2.0)
    kappa[0, 0, 1] = 4.0
    ax, ay, az = F.face_acceleration(grid, C, kappa, 0.5, (0.1, 0.2, -0.3), 3.0, 1.0)
    assert ax.shape == (2, 2, 2) and ay.shape == (2, 2, 2) and az.shape == (3, 2, 2)
    np.testing.assert_allclose(ax[0, 0, 1], -0.65, rtol=1e-15)
    np.testing.assert_allclose(ax[0, 0, 0], 0.85, rtol=1e-15)
    np.testing.assert_allclose(ax[1, 0, 1], 0.1, rtol=1e-15)
    np.testing.assert_allclose(ay[0, 0, 0], -0.2, rtol=1e-14)
    np.testing.assert_allclose(ay[0, 1, 0], 0.6, rtol=1e-15)
    np.testing.assert_allclose(az[1, 0, 0], 0.1, rtol=1e-14)
    np.testing.assert_allclose(az[1, 0, 1], 9.0 / 7.0 - 0.3, rtol=1e-15)
    assert np.all(az[0] == 0.0) and np.all(az[2] == 0.0)


def test_predictor_adds_tau_a_and_zeroes_walls():
    grid = pi.Grid(5, 4, 3, 0.2, (W, P, W))
    pr = pi.random_problem(grid, seed=21)
    un = [x.copy() for x in (pr.u, pr.v, pr.w)]
    un[0][:, :, 0] = un[0][:, :, -1] = 5.0  # u^n on the wall faces is not carried over
    un[2][0] = un[2][-1] = -5.0
    kappa = pi.random_field(grid.shape, seed=22, mean_free=False)
    acc = F.face_acceleration(grid, pr.C, kappa, 0.07, (0.0, -1.0, 2.0), pr.rho1, pr.rho2)
    us = F.predictor(grid, *un, pr.C, kappa, 0.07, (0.0, -1.0, 2.0), pr.rho1, pr.rho2, 0.01)
    for axis in range(3):
        want = un[axis] + 0.01 * acc[axis]
        if grid.bc[axis] == W:
            sl = [slice(None)] * 3
            for end in (0, -1):
                sl[2 - axis] = end
                want[tuple(sl)] = 0.0
        np.testing.assert_array_equal(us[axis], want)
    assert np.all(us[0][:, :, 0] == 0.0) and np.all(us[2][-1] == 0.0)


def _project(grid, C, rho1, rho2, tau, ustar):
    return oracle.projection_step(grid, C, rho1, rho2, tau, *ustar, tol=1e-14)


@pytest.mark.parametrize("bc", [(P, P, P), (P, P, W), (W, P, W)])
@pytest.mark.parametrize("kappa", [-8.0, 3.0])
def test_constant_curvature_is_well_balanced(bc, kappa):
    """Constant kappa, no gravity, u^n = 0, density ratio 1000: u* = tau beta grad(-sigma kappa C)
    is a discrete gradient with the projection's weights, so the projection (dt = tau)
    returns p = -sigma kappa (C - mean C) and u = 0 (no spurious currents)."""
    grid = pi.Grid(24, 20, 16, 1.0 / 24, bc)
    pr = pi.random_problem(grid, seed=23, rho1=1000.0, drops=3)
    sigma, tau = 0.07, 1e-3
    z = [np.zeros(grid.face_shape(a)) for a in range(3)]
    ustar = F.predictor(grid, *z, pr.C, kappa, sigma, (0.0, 0.0, 0.0), pr.rho1, pr.rho2, tau)
    res = _project(grid, pr.C, pr.rho1, pr.rho2, tau, ustar)
    phi = -sigma * kappa * (pr.C - pr.C.mean())
    lmin, lmax = res.cg.lanczos_extremes()
    err = np.linalg.norm(res.p - phi)
    assert err <= (lmax / lmin) * max(res.cg.rel_res_l2, 1e-16) * np.linalg.norm(phi) + 1e-13 * np.linalg.norm(phi)
    assert err <= 1e-8 * np.linalg.norm(phi)
    umax = max(np.abs(x).max() for x in ustar)
    assert umax > 0
    for uu in res.u:
        assert np.abs(uu).max() <= 1e-8 * umax


def test_laplace_pressure_jump_of_a_drop():
    """A sphere of fluid 1, radius R, kappa = -2/R (the sign convention that makes
    Eq. csf2 agree with Eq. jump1): the projected pressure inside exceeds the
    pressure far outside by 2 sigma / R (Laplace)."""
    n, R, sigma, tau = 32, 0.25, 0.07, 1e-3
    grid = pi.Grid(n, n, n, 1.0 / n, (P, P, P))
    C = np.zeros(grid.shape)
    pi.add_sphere(C, grid, (0.5, 0.5, 0.5), R)
    z = [np.zeros(grid.face_shape(a)) for a in range(3)]
    ustar = F.predictor(grid, *z, C, -2.0 / R, sigma, (0.0, 0.0, 0.0), 10.0, 1.0, tau)
    res = _project(grid, C, 10.0, 1.0, tau, ustar)
    jump = res.p[n // 2, n // 2, n // 2] - res.p[0, 0, 0]
    assert C[n // 2, n // 2, n // 2] == 1.0 and C[0, 0, 0] == 0.0
    assert abs(jump - 2.0 * sigma / R) <= 1e-9 * 2.0 * sigma / R


def test_hydrostatic_balance_of_a_layered_fluid():
    """Heavy fluid below a flat interface, walls in z, gravity -g e_z, plus a constant
    curvature: u* = tau a_f is the face gradient (weights beta_f) of the discrete
    hydrostatic pressure p_{k+1} = p_k - g h (rho_k + rho_{k+1})/2 plus -sigma kappa C,
    so the projection returns that pressure (mean-free) and u = 0."""
    nz, h = 32, 1.0 / 32
    grid = pi.Grid(8, 6, nz, h, (P, P, W))
    zc = (np.arange(nz) + 0.5) * h
    frac = np.clip((0.41 - (zc - h / 2)) / h, 0.0, 1.0)  # fraction of each cell below z = 0.41
    C = np.broadcast_to(frac[:, None, None], grid.shape).copy()
    rho1, rho2, g, sigma, kappa, tau = 1000.0, 1.2, 9.81, 0.07, 3.0, 1e-3
    z = [np.zeros(grid.face_shape(a)) for a in range(3)]
    ustar = F.predictor(grid, *z, C, kappa, sigma, (0.0, 0.0, -g), rho1, rho2, tau)
    res = _project(grid, C, rho1, rho2, tau, ustar)
    rho = rho1 * frac + rho2 * (1.0 - frac)
    ph = np.zeros(nz)
    for k in range(nz - 1):
        ph[k + 1] = ph[k] - g * h * (rho[k] + rho[k + 1]) / 2.0
    p = ph - sigma * kappa * frac
    want = np.broadcast_to((p - p.mean())[:, None, None], grid.shape)
    scale = np.abs(want).max()
    assert np.abs(res.p - want).max() <= 1e-9 * scale
    umax = tau * g
    for uu in res.u:
        assert np.abs(uu).max() <= 1e-8 * umax


@pytest.mark.parametrize("rho_drop, rho_around, rises", [(1.0, 1000.0, True), (1000.0, 1.0, False)])
def test_buoyancy_sign(rho_drop, rho_around, rises):
    """Gravity -g e_z on a drop of fluid 1 in fluid 2 (walls in z): after the
    projection the velocity through the drop's centre points up for a light drop
    and down for a heavy one (Archimedes)."""
    n = 16
    grid = pi.Grid(n, n, n, 1.0 / n, (P, P, W))
    C = np.zeros(grid.shape)
    pi.add_sphere(C, grid, (0.5, 0.5, 0.5), 0.2)
    z = [np.zeros(grid.face_shape(a)) for a in range(3)]
    ustar = F.predictor(grid, *z, C, 0.0, 0.0, (0.0, 0.0, -9.81), rho_drop, rho_around, 1e-3)
    res = _project(grid, C, rho_drop, rho_around, 1e-3, ustar)
    wc = res.u[2][n // 2, n // 2, n // 2]  # z-face through the centre
    assert (wc > 0) == rises and abs(wc) > 1e-6
