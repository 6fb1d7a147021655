"""Pins of the solid-cell oracle (oracle/solid.py, Sec. 3.8 "Solid
boundaries") against what the paper and the mathematics fix, on the CPU.

Each test names the mistake it would catch: a link flag taken from one cell
only, a solid that leaks flux, a gauge over the wrong cells, a null-space
projection that drifts."""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle
import paris_inputs as pi
from oracle import solid as S

P, W = pi.PERIODIC, pi.WALL


def test_face_flags_around_one_solid_cell():
    """3x3x3 periodic box, cell (1,1,1) solid: exactly its six faces are
    closed; a link flag taken from one side only (the printed loop read
    literally) would leave three of them open."""
    g = pi.Grid(3, 3, 3, 1 / 3)
    fl = np.ones(g.shape, np.uint8)
    fl[1, 1, 1] = 0
    sx, sy, sz = S.face_flags(g, fl)
    closed = {(0, 1, 1, 1), (0, 1, 1, 2), (1, 1, 1, 1), (1, 1, 2, 1), (2, 1, 1, 1), (2, 2, 1, 1)}
    for axis, f in enumerate((sx, sy, sz)):
        for k in range(3):
            for j in range(3):
                for i in range(3):
                    want = 0.0 if (axis, k, j, i) in closed else 1.0
                    assert f[k, j, i] == want, (axis, k, j, i)


def test_wall_faces_are_closed():
    g = pi.Grid(4, 3, 5, 0.25, (W, P, W))
    sx, sy, sz = S.face_flags(g, np.ones(g.shape, np.uint8))
    assert sx.shape == (5, 3, 5) and sz.shape == (6, 3, 4)
    assert np.all(sx[:, :, 0] == 0) and np.all(sx[:, :, -1] == 0) and np.all(sx[:, :, 1:-1] == 1)
    assert np.all(sy == 1)
    assert np.all(sz[0] == 0) and np.all(sz[-1] == 0) and np.all(sz[1:-1] == 1)


@pytest.mark.parametrize("grid", [pi.Grid(12, 10, 8, 1 / 12), pi.Grid(9, 8, 11, 0.1, (W, P, W))],
                         ids=["ppp", "wpw"])
def test_no_solid_is_the_plain_projection(grid):
    """All cells fluid: the masked projection is the plain one."""
    pr = pi.random_problem(grid, seed=71)
    ref = oracle.projection_step(grid, pr.C, pr.rho1, pr.rho2, pr.dt, pr.u, pr.v, pr.w)
    p, u, beta, res, _ = S.projection_step_solid(grid, pr.C, pr.rho1, pr.rho2, pr.dt, pr.u, pr.v, pr.w,
                                                 np.ones(grid.shape, np.uint8))
    assert np.abs(p - ref.p).max() <= 1e-10 * np.abs(ref.p).max()
    for a in range(3):
        assert np.abs(u[a] - ref.u[a]).max() <= 1e-10 * max(np.abs(ref.u[a]).max(), 1.0)


def test_solid_slab_equals_a_wall_pair():
    """A periodic-z box whose planes 4 and 5 are solid is the walls-in-z box
    of the remaining planes 6..11, 0..3 (in that order): same p on the fluid
    cells and same velocity on the corresponding faces."""
    nz, k_lo, k_hi = 12, 4, 5
    g = pi.Grid(10, 8, nz, 1 / 10, (P, P, P))
    pr = pi.random_problem(g, seed=72, rho1=200.0)
    fl = np.ones(g.shape, np.uint8)
    fl[k_lo:k_hi + 1] = 0
    order = [(k_hi + 1 + m) % nz for m in range(nz - (k_hi - k_lo + 1))]
    gw = pi.Grid(10, 8, len(order), 1 / 10, (P, P, W))
    Cw = pr.C[order]
    uw, vw = pr.u[order], pr.v[order]
    ww = np.zeros(gw.face_shape(2))
    for m in range(1, len(order)):  # wall-grid face m lies between planes order[m-1] and order[m]
        ww[m] = pr.w[order[m]]
    ref = oracle.projection_step(gw, Cw, pr.rho1, pr.rho2, pr.dt, uw, vw, ww)
    p, u, _, res, _ = S.projection_step_solid(g, pr.C, pr.rho1, pr.rho2, pr.dt, pr.u, pr.v, pr.w, fl)
    assert res.rel_res_l2 <= 1e-12
    assert np.all(p[k_lo:k_hi + 1] == 0.0)
    scale = np.abs(ref.p).max()
    assert np.abs(p[order] - ref.p).max() <= 1e-9 * scale
    assert np.abs(u[0][order] - ref.u[0]).max() <= 1e-9 * np.abs(ref.u[0]).max()
    assert np.abs(u[1][order] - ref.u[1]).max() <= 1e-9 * np.abs(ref.u[1]).max()
    for m in range(1, len(order)):
        assert np.abs(u[2][order[m]] - ref.u[2][m]).max() <= 1e-9 * np.abs(ref.u[2]).max()
    assert np.all(u[2][k_lo:k_hi + 2] == 0.0)  # the faces into and inside the slab


def _bordered_solve(grid, beta, b, fluid):
    """Dense solve of -L p = -b on the fluid cells with sum(p) = 0 (a
    Lagrange multiplier): the plain definition, by numpy.linalg.solve."""
    op = oracle.Operator(grid, *beta)
    rowptr, col, val = op.csr()
    op.close()
    A = sp.csr_matrix((val, col, rowptr), shape=(grid.ncells, grid.ncells)).toarray()
    f = fluid.ravel().astype(bool)
    Aff = A[np.ix_(f, f)]
    n = Aff.shape[0]
    M = np.zeros((n + 1, n + 1))
    M[:n, :n] = Aff
    M[:n, n] = 1.0
    M[n, :n] = 1.0
    rhs = np.concatenate([-b.ravel()[f], [0.0]])
    sol = np.linalg.solve(M, rhs)
    p = np.zeros(grid.ncells)
    p[f] = sol[:n]
    return p.reshape(grid.shape)


@pytest.mark.parametrize("grid", [pi.Grid(6, 6, 6, 1 / 6), pi.Grid(7, 5, 6, 0.2, (W, P, W))], ids=["ppp", "wpw"])
def test_interior_block_against_dense_solve(grid):
    """An interior solid block: p equals the dense bordered solve on the fluid
    cells, the faces around the block carry no velocity, and the corrected
    velocity is divergence-free in every fluid cell."""
    pr = pi.random_problem(grid, seed=73, rho1=1000.0)
    fl = np.ones(grid.shape, np.uint8)
    fl[2:4, 1:3, 2:4] = 0
    p, u, beta, res, b = S.projection_step_solid(grid, pr.C, pr.rho1, pr.rho2, pr.dt, pr.u, pr.v, pr.w, fl)
    pd = _bordered_solve(grid, beta, oracle.null_project(b, fl), fl)
    assert np.abs(p - pd).max() <= 1e-9 * np.abs(pd).max()
    flags = S.face_flags(grid, fl)
    for a in range(3):
        assert np.all(u[a][flags[a] == 0] == 0.0)
    d = oracle.divergence(grid, *u, dt=1.0)
    umax = max(np.abs(x).max() for x in (pr.u, pr.v, pr.w))
    assert np.abs(d[fl == 1]).max() <= 1e-9 * umax / grid.h
    assert np.all(d[fl == 0] == 0.0)


def test_gradient_field_with_a_solid_is_recovered():
    """u* = dt B_s G phi with the masked coefficients: p = phi on the fluid
    cells (up to the fluid mean), u = 0 everywhere, for any density ratio."""
    g = pi.Grid(16, 12, 10, 1 / 16, (P, P, W))
    pr = pi.random_problem(g, seed=74, rho1=1000.0)
    fl = np.ones(g.shape, np.uint8)
    fl[3:6, 4:8, 5:9] = 0
    beta = S.face_coeffs_solid(g, pr.C, pr.rho1, pr.rho2, fl)
    phi = pi.random_field(g.shape, seed=75)
    gx, gy, gz = oracle.face_gradient(g, phi)
    us = [pr.dt * b * gr for b, gr in zip(beta, (gx, gy, gz))]
    p, u, _, res, _ = S.projection_step_solid(g, pr.C, pr.rho1, pr.rho2, pr.dt, *us, fl)
    want = oracle.null_project(phi, fl)
    assert np.abs(p - want).max() <= 1e-8 * np.abs(want).max()
    umax = max(np.abs(x).max() for x in us)
    assert max(np.abs(x).max() for x in u) <= 1e-8 * umax
