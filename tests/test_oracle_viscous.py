"""Pins of the implicit viscous oracle (Eq. muelliptic, oracle/viscous.py)
against closed forms, brute force and a manufactured solution (CPU)."""
import numpy as np
import pytest
import scipy.fft as sfft

import paris_inputs as pi
from oracle import viscous as V

P, W = pi.PERIODIC, pi.WALL


def _lam(m, h, kind):
    """eigenvalues of the 1-D second difference (negative), in the order the
    matching transform returns its coefficients"""
    k = np.arange(m)
    if kind == "periodic":
        return -4.0 / h**2 * np.sin(np.pi * k / m) ** 2
    if kind == "dirichlet":  # DST-I, modes k = 1..m on m interior points of m+1 intervals
        return -4.0 / h**2 * np.sin(np.pi * (k + 1) / (2 * (m + 1))) ** 2
    return -4.0 / h**2 * np.sin(np.pi * (k + 1) / (2 * m)) ** 2  # noslip: DST-II, modes 1..m


def _closed_form(grid, comp, nu, tau, un):
    """u* for constant nu by diagonalising each axis' second difference"""
    shape = V.unknown_shape(grid, comp)
    kinds, lam = [], []
    for axis in range(3):
        m = shape[2 - axis]
        kind = "periodic" if grid.bc[axis] == P else ("dirichlet" if axis == comp else "noslip")
        kinds.append(kind)
        lam.append(_lam(m, grid.h, kind))
    c = np.asarray(un, dtype=np.complex128)
    for axis, kind in enumerate(kinds):
        ax = 2 - axis
        if kind == "periodic":
            c = sfft.fft(c, axis=ax)
        elif kind == "dirichlet":
            c = sfft.dst(c.real, type=1, axis=ax) + 1j * sfft.dst(c.imag, type=1, axis=ax)
        else:
            c = sfft.dst(c.real, type=2, axis=ax) + 1j * sfft.dst(c.imag, type=2, axis=ax)
    L = lam[2][:, None, None] + lam[1][None, :, None] + lam[0][None, None, :]
    c = c / (1.0 - tau * nu * L)
    for axis, kind in reversed(list(enumerate(kinds))):
        ax = 2 - axis
        if kind == "periodic":
            c = sfft.ifft(c, axis=ax)
        elif kind == "dirichlet":
            c = sfft.idst(c.real, type=1, axis=ax) + 1j * sfft.idst(c.imag, type=1, axis=ax)
        else:
            c = sfft.idst(c.real, type=2, axis=ax) + 1j * sfft.idst(c.imag, type=2, axis=ax)
    return c.real


CASES = [(pi.Grid(8, 6, 10, 0.1, (P, P, P)), 0), (pi.Grid(8, 6, 10, 0.1, (P, P, P)), 2),
         (pi.Grid(8, 6, 10, 0.1, (P, P, W)), 2), (pi.Grid(8, 6, 10, 0.1, (P, P, W)), 0),
         (pi.Grid(6, 8, 5, 0.2, (W, P, W)), 0), (pi.Grid(6, 8, 5, 0.2, (W, W, W)), 1),
         (pi.Grid(6, 8, 5, 0.2, (W, W, W)), 2)]


@pytest.mark.parametrize("grid,comp", CASES, ids=lambda x: str(x) if isinstance(x, int) else
                         f"{x.nx}x{x.ny}x{x.nz}_{''.join('pw'[b] for b in x.bc)}")
def test_constant_viscosity_matches_transform_closed_form(grid, comp):
    """Constant nu: each axis' second difference is diagonalised by the FFT
    (periodic), the DST-I (normal component at walls, zero on the wall faces)
    or the DST-II (tangential component, no-slip half a cell from the wall)."""
    rng = np.random.default_rng([7, comp])
    un = rng.standard_normal(V.unknown_shape(grid, comp))
    nu, tau = 0.37, 0.05
    us = V.solve(grid, comp, np.full(un.shape, nu), tau, un)
    ref = _closed_form(grid, comp, nu, tau, un)
    assert np.max(np.abs(us - ref)) <= 1e-11 * np.max(np.abs(ref))


def test_zero_time_step_returns_the_input():
    grid = pi.Grid(6, 6, 6, 0.1, (P, W, P))
    un = np.random.default_rng(1).standard_normal(V.unknown_shape(grid, 1))
    assert np.array_equal(V.solve(grid, 1, np.ones(un.shape), 0.0, un), un)


def _brute_laplacian(grid, comp):
    """the Laplacian entry by entry from the neighbour rules (dense)"""
    shape = V.unknown_shape(grid, comp)
    nz, ny, nx = shape
    n = nx * ny * nz
    A = np.zeros((n, n))
    idx = lambda i, j, k: (k * ny + j) * nx + i
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                r = idx(i, j, k)
                for axis, (pos, m) in enumerate(((i, nx), (j, ny), (k, nz))):
                    for step in (-1, 1):
                        A[r, r] -= 1.0
                        q = pos + step
                        if 0 <= q < m:
                            nb = [i, j, k]
                            nb[axis] = q
                            A[r, idx(*nb)] += 1.0
                        elif grid.bc[axis] == P:
                            nb = [i, j, k]
                            nb[axis] = q % m
                            A[r, idx(*nb)] += 1.0
                        elif axis == comp:
                            pass  # the wall face: u = 0
                        else:
                            A[r, r] -= 1.0  # beyond a no-slip wall: minus the value here
    return A / grid.h**2


@pytest.mark.parametrize("bc,comp", [((P, P, W), 0), ((P, P, W), 2), ((W, P, W), 1), ((W, W, W), 0),
                                     ((P, P, P), 1)])
def test_laplacian_matches_brute_force(bc, comp):
    grid = pi.Grid(4, 3, 5, 0.5, bc)
    L = V.laplacian(grid, comp).toarray()
    np.testing.assert_array_equal(L, _brute_laplacian(grid, comp))


def test_spd_form_is_symmetric_and_positive_definite():
    grid = pi.Grid(5, 4, 6, 0.25, (W, P, W))
    rng = np.random.default_rng(3)
    for comp in range(3):
        nu = rng.uniform(0.01, 2.0, V.unknown_shape(grid, comp))
        A = V.spd_operator(grid, comp, nu, 0.1).toarray()
        assert np.array_equal(A, A.T)
        assert np.linalg.eigvalsh(A).min() > 0.0


def test_face_viscosity_is_the_ratio_of_face_means():
    grid = pi.Grid(3, 2, 2, 1.0, (W, P, P))
    C = np.zeros(grid.shape)
    C[:, :, 1] = 1.0  # the middle column is fluid 1
    nu_x = V.face_nu(grid, 0, C, 2.0, 0.5, 10.0, 1.0)  # interior x-faces 1, 2
    # face 1: cells 0 (fluid 2: mu 0.5, rho 1) and 1 (fluid 1: mu 2, rho 10)
    np.testing.assert_allclose(nu_x[..., 0], (0.5 + 2.0) / (1.0 + 10.0), rtol=0, atol=0)
    np.testing.assert_allclose(nu_x[..., 1], (2.0 + 0.5) / (10.0 + 1.0), rtol=0, atol=0)
    nu_y = V.face_nu(grid, 1, C, 2.0, 0.5, 10.0, 1.0)  # periodic: both sides in the same column
    np.testing.assert_array_equal(nu_y[:, :, 1], np.full((2, 2), 2.0 / 10.0))
    np.testing.assert_array_equal(nu_y[:, :, 0], np.full((2, 2), 0.5 / 1.0))


def test_variable_viscosity_solution_satisfies_the_equation():
    grid = pi.Grid(10, 8, 12, 1 / 12, (P, W, W))
    rng = np.random.default_rng(5)
    C = (rng.random(grid.shape) < 0.3).astype(float)
    for comp in range(3):
        nu = V.face_nu(grid, comp, C, 1e-2, 1e-4, 1000.0, 1.0)
        un = rng.standard_normal(V.unknown_shape(grid, comp))
        us = V.solve(grid, comp, nu, 1e-3, un)
        r = V.residual(grid, comp, nu, 1e-3, us, un)
        assert np.max(np.abs(r)) <= 1e-11 * np.max(np.abs(un))


def test_manufactured_solution_converges_at_second_order():
    """u = sin(pi z) cos(2 pi x) cos(2 pi y), zero on the z-walls (no-slip),
    nu = 1 + 0.5 sin(2 pi x): u^n = u - tau nu Lap u analytically; the error
    of u* falls by about 4 per halving of h (x component, staggered in x)."""
    tau, errs = 0.01, []
    for n in (16, 32, 64):
        h = 1.0 / n
        grid = pi.Grid(n, n, n, h, (P, P, W))
        x = np.arange(n) * h  # x-faces at i h
        yc = (np.arange(n) + 0.5) * h
        zc = (np.arange(n) + 0.5) * h
        Z, Y, X = np.meshgrid(zc, yc, x, indexing="ij")
        u = np.sin(np.pi * Z) * np.cos(2 * np.pi * X) * np.cos(2 * np.pi * Y)
        lap = -(np.pi**2 + 8 * np.pi**2) * u
        nu = 1.0 + 0.5 * np.sin(2 * np.pi * X)
        us = V.solve(grid, 0, nu, tau, u - tau * nu * lap)
        errs.append(np.max(np.abs(us - u)))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.4 < r1 < 4.6 and 3.4 < r2 < 4.6, errs


def test_solve_reports_its_iterations():
    grid = pi.Grid(8, 6, 4, 0.125, (P, W, P))
    nu = np.full(V.unknown_shape(grid, 1), 1e-2)
    un = np.random.default_rng(6).standard_normal(nu.shape)
    info = {}
    V.solve(grid, 1, nu, 0.1, un, stats=info)
    assert info["iters"] >= 1
    V.solve(grid, 1, nu, 0.0, un, stats=info)
    assert info["iters"] == 0


def test_viscous_golden_matches_its_inputs():
    """The stored 256^3 oracle solves (golden/viscous256_drops.json) belong to
    the current input generator and parameters, converged, and obey the
    discrete maximum-norm bound |u*| <= tau max(nu) max|u^n/(tau nu)| of a
    strictly diagonally dominant SPD form with margin 1/(tau nu)."""
    import hashlib
    import json
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "viscous256_drops.json")
    if not os.path.exists(path):
        pytest.skip("golden/viscous256_drops.json not generated")
    with open(path) as fh:
        gold = json.load(fh)
    pr = pi.config2(n=256)
    g = pr.grid
    assert hashlib.sha256(np.ascontiguousarray(pr.C).tobytes()).hexdigest() == gold["C_sha256"]
    nus = [V.face_nu(g, c, pr.C, gold["mu1"], gold["mu2"], pr.rho1, pr.rho2) for c in range(3)]
    tau = gold["tau_nu_over_h2"] * g.h ** 2 / max(float(nu.max()) for nu in nus)
    assert tau == gold["tau"]
    for c, rec in enumerate(gold["components"]):
        n = int(np.prod(V.unknown_shape(g, c)))
        assert rec["rel_res_l2"] <= 1e-12 and rec["rel_res_linf"] <= 1e-12 and rec["iters"] > 0
        idx = np.asarray(rec["unknowns"])
        assert idx.min() >= 0 and idx.max() < n and len(rec["x"]) == len(idx)
        un = V.interior(g, c, (pr.u, pr.v, pr.w)[c])
        bound = tau * nus[c].max() * np.abs(un / (tau * nus[c])).max()
        assert np.abs(rec["x"]).max() <= rec["x_max_abs"] <= bound * (1 + 1e-12)
