"""Parity of the implicit viscous step (Sec. 3.2.3, Eq. muelliptic) on the GPU,
through the C ABI, with the FP64 CPU oracle (oracle/viscous.py).

Bars: the face viscosity is bitwise (both sides round each product and sum in
the same order); the solve must meet its own stopping test when the residual
of the SPD form is recomputed by the oracle (relative L2 and L-infinity norms
<= 1e-11 for tol = 1e-12), and agree with the oracle's solution to
||u* - u*_oracle||_inf / ||u*_oracle||_inf <= 1e-9: the SPD form's condition
number here stays below 1e3, so residuals of 1e-12 bound the error near 1e-9.
Wall faces of the component are filled with NaN on input (never read) and must
come back 0.
"""
import hashlib
import json
import os

import numpy as np
import pytest

import paris_inputs as pi
from oracle import viscous as V

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
P, W = pi.PERIODIC, pi.WALL
MU1, MU2, RHO1, RHO2 = 1.0e-3, 1.8e-5, 1000.0, 1.2  # water-like and air-like phases


@pytest.fixture(scope="module")
def paris():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2012_11744_gb300 as m
    m.build()
    return m


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def host(t):
    return t.detach().cpu().numpy()


GRIDS = [
    pi.Grid(16, 16, 16, 1 / 16, (P, P, P)),
    pi.Grid(24, 20, 16, 1 / 24, (P, P, W)),
    pi.Grid(17, 9, 12, 0.05, (W, P, W)),
    pi.Grid(6, 5, 3, 0.2, (W, W, W)),
    pi.Grid(2, 2, 2, 0.5, (W, W, W)),
    pi.Grid(48, 2, 10, 1 / 48, (P, W, P)),
    pi.Grid(64, 64, 64, 1 / 64, (P, P, W)),
]
GID = [f"{g.nx}x{g.ny}x{g.nz}_{''.join('pw'[b] for b in g.bc)}" for g in GRIDS]


def _walls(grid, comp):
    """mask of the component's wall faces in its full face array"""
    return V.embed(grid, comp, np.ones(V.unknown_shape(grid, comp))) == 0


def _problem(grid, comp, seed):
    pr = pi.random_problem(grid, seed=seed)
    nu = V.face_nu(grid, comp, pr.C, MU1, MU2, RHO1, RHO2)
    # tau with max tau nu / h^2 = 20: the Laplacian dominates in the light phase
    tau = 20.0 * grid.h ** 2 / nu.max()
    un = V.interior(grid, comp, (pr.u, pr.v, pr.w)[comp])
    un = un + 0.1 * np.random.default_rng([300, seed, comp]).standard_normal(un.shape)
    return pr, nu, tau, un


def _full(grid, comp, interior_values):
    a = V.embed(grid, comp, interior_values)
    a[_walls(grid, comp)] = np.nan
    return a


@pytest.mark.parametrize("grid", GRIDS, ids=GID)
@pytest.mark.parametrize("comp", [0, 1, 2])
def test_face_viscosity_matches_oracle(paris, grid, comp):
    pr = pi.random_problem(grid, seed=11)
    ref = V.face_nu(grid, comp, pr.C, MU1, MU2, RHO1, RHO2)
    with paris.Context(grid) as ctx:
        got = host(ctx.face_viscosity(comp, dev(pr.C), MU1, MU2, RHO1, RHO2))
    np.testing.assert_array_equal(V.interior(grid, comp, got), ref)
    assert np.all(got[_walls(grid, comp)] == 0.0)


@pytest.mark.parametrize("multigrid", [False, True], ids=["jacobi", "mg"])
@pytest.mark.parametrize("grid", GRIDS, ids=GID)
@pytest.mark.parametrize("comp", [0, 1, 2])
def test_viscous_solve_matches_oracle(paris, grid, comp, multigrid):
    pr, nu, tau, un = _problem(grid, comp, seed=12)
    ref = V.solve(grid, comp, nu, tau, un)
    with paris.Context(grid) as ctx:
        us, st = ctx.viscous_solve(comp, dev(_full(grid, comp, nu)), tau, dev(_full(grid, comp, un)),
                                   tol=1e-12, multigrid=multigrid)
        us = host(us)
    assert st["converged"] == 1 and st["iters"] >= 1
    assert np.all(us[_walls(grid, comp)] == 0.0)
    x = V.interior(grid, comp, us)
    A = V.spd_operator(grid, comp, nu, tau)
    b = (un / (tau * nu)).ravel()
    res = b - A @ x.ravel()
    assert np.linalg.norm(res) <= 1e-11 * np.linalg.norm(b)
    assert np.abs(res).max() <= 1e-11 * np.abs(b).max()
    assert np.abs(x - ref).max() <= 1e-9 * np.abs(ref).max()
    # the equation as printed holds too
    r = V.residual(grid, comp, nu, tau, x, un)
    assert np.abs(r).max() <= 1e-9 * np.abs(un).max()


def test_viscous_solve_from_the_context_coefficients(paris):
    """face viscosity from the GPU feeding the GPU solve, all three components"""
    grid = pi.Grid(32, 24, 16, 1 / 32, (W, P, W))
    pr = pi.random_problem(grid, seed=13)
    with paris.Context(grid) as ctx:
        for comp in range(3):
            nu_d = ctx.face_viscosity(comp, dev(pr.C), MU1, MU2, RHO1, RHO2)
            nu = V.interior(grid, comp, host(nu_d))
            tau = 5.0 * grid.h ** 2 / nu.max()
            un = V.interior(grid, comp, (pr.u, pr.v, pr.w)[comp])
            us, st = ctx.viscous_solve(comp, nu_d, tau, dev(_full(grid, comp, un)), tol=1e-12)
            ref = V.solve(grid, comp, nu, tau, un)
            x = V.interior(grid, comp, host(us))
            assert st["converged"] == 1
            assert np.abs(x - ref).max() <= 1e-9 * np.abs(ref).max()


def test_viscous_tau_zero_returns_un(paris):
    grid = pi.Grid(9, 7, 5, 0.1, (P, W, W))
    pr, nu, _, un = _problem(grid, 1, seed=14)
    with paris.Context(grid) as ctx:
        us, st = ctx.viscous_solve(1, dev(_full(grid, 1, nu)), 0.0, dev(_full(grid, 1, un)))
        us = host(us)
    assert st["converged"] == 1 and st["iters"] == 0
    np.testing.assert_array_equal(V.interior(grid, 1, us), un)
    assert np.all(us[_walls(grid, 1)] == 0.0)


def test_viscous_zero_right_hand_side(paris):
    grid = pi.Grid(8, 8, 8, 0.125, (W, W, W))
    shp = V.unknown_shape(grid, 2)
    nu = np.full(shp, 1e-3)
    with paris.Context(grid) as ctx:
        us, st = ctx.viscous_solve(2, dev(_full(grid, 2, nu)), 1.0, dev(_full(grid, 2, np.zeros(shp))))
        us = host(us)
    assert st["converged"] == 1 and st["iters"] == 0
    assert np.all(us == 0.0)


def test_viscous_errors(paris):
    import ctypes as ct
    from paper_2012_11744_gb300 import _abi
    grid = pi.Grid(8, 6, 4, 0.125, (P, W, P))
    pr, nu, tau, un = _problem(grid, 0, seed=15)
    with paris.Context(grid) as ctx:
        nu_d, un_d = dev(_full(grid, 0, nu)), dev(_full(grid, 0, un))
        us = torch.empty_like(un_d)
        lib, p = ctx.lib, ctx._ptr
        ptr = lambda t: ct.c_void_p(t.data_ptr())  # noqa: E731
        call = lambda comp, nu_, t, un_, us_, tol, it: lib.paris_viscous_solve(  # noqa: E731
            p, comp, nu_, t, un_, us_, tol, it, None)
        assert call(3, ptr(nu_d), tau, ptr(un_d), ptr(us), 1e-10, 10) == 1
        assert call(0, ptr(nu_d), -1.0, ptr(un_d), ptr(us), 1e-10, 10) == 1
        assert call(0, ptr(nu_d), float("nan"), ptr(un_d), ptr(us), 1e-10, 10) == 1
        assert call(0, ptr(nu_d), tau, ptr(un_d), ptr(un_d), 1e-10, 10) == 1
        assert call(0, ptr(nu_d), tau, ptr(un_d), ptr(us), 1.0, 10) == 1
        assert call(0, ptr(nu_d), tau, ptr(un_d), ptr(us), 1e-10, 0) == 1
        assert call(0, None, tau, ptr(un_d), ptr(us), 1e-10, 10) == 1
        # a viscosity that is not positive on an unknown
        bad = nu.copy()
        bad[1, 2, 3] = 0.0
        assert call(0, ptr(dev(_full(grid, 0, bad))), tau, ptr(un_d), ptr(us), 1e-10, 10) == 4
        # too few iterations: the last iterate comes back
        st = _abi.Stats()
        s = lib.paris_viscous_solve(p, 0, ptr(nu_d), tau, ptr(un_d), ptr(us), 1e-14, 2, ct.byref(st))
        assert s == 3 and st.iters == 2 and st.converged == 0
        assert lib.paris_face_viscosity(p, 0, ptr(dev(pr.C)), 0.0, MU2, RHO1, RHO2, ptr(us)) == 1
        assert lib.paris_face_viscosity(p, -1, ptr(dev(pr.C)), MU1, MU2, RHO1, RHO2, ptr(us)) == 1


@pytest.mark.parametrize("tnu", [4.0, 40.0, 400.0])
@pytest.mark.parametrize("comp", [0, 2])
def test_multigrid_needs_few_iterations(paris, comp, tnu):
    """64^3 drop field with walls in z (the 256^3 recipe), tau nu/h^2 = tnu:
    the V-cycle-preconditioned solve meets tol 1e-10 in at most 10 iterations
    where Jacobi-PCG needs tens to hundreds, and both reach the same u*."""
    pr = pi.config2(n=64)
    g = pr.grid
    with paris.Context(g) as ctx:
        C = dev(pr.C)
        nu_d = ctx.face_viscosity(comp, C, MU1, MU2, pr.rho1, pr.rho2)
        tau = tnu * g.h ** 2 / float(nu_d.max())
        un = dev((pr.u, pr.v, pr.w)[comp])
        um, sm = ctx.viscous_solve(comp, nu_d, tau, un, tol=1e-10, multigrid=True)
        uj, sj = ctx.viscous_solve(comp, nu_d, tau, un, tol=1e-10, max_iter=5000)
        assert sm["converged"] == 1 and sj["converged"] == 1
        assert sm["iters"] <= 10, sm
        assert sj["iters"] > 2 * sm["iters"], (sj, sm)
        a, b = V.interior(g, comp, host(um)), V.interior(g, comp, host(uj))
        assert np.abs(a - b).max() <= 1e-8 * np.abs(b).max()


def test_viscous_mg_errors(paris):
    import ctypes as ct
    from paper_2012_11744_gb300 import _abi
    grid = pi.Grid(8, 6, 4, 0.125, (P, W, P))
    pr, nu, tau, un = _problem(grid, 0, seed=15)
    with paris.Context(grid) as ctx:
        nu_d, un_d = dev(_full(grid, 0, nu)), dev(_full(grid, 0, un))
        us = torch.empty_like(un_d)
        lib, p = ctx.lib, ctx._ptr
        ptr = lambda t: ct.c_void_p(t.data_ptr())  # noqa: E731
        call = lambda comp, nu_, t, un_, us_, tol, it: lib.paris_viscous_solve_mg(  # noqa: E731
            p, comp, nu_, t, un_, us_, tol, it, None)
        assert call(3, ptr(nu_d), tau, ptr(un_d), ptr(us), 1e-10, 10) == 1
        assert call(0, ptr(nu_d), -1.0, ptr(un_d), ptr(us), 1e-10, 10) == 1
        assert call(0, ptr(nu_d), tau, ptr(un_d), ptr(un_d), 1e-10, 10) == 1
        assert call(0, ptr(nu_d), tau, ptr(un_d), ptr(us), 1e-10, 0) == 1
        bad = nu.copy()
        bad[1, 2, 3] = 0.0
        assert call(0, ptr(dev(_full(grid, 0, bad))), tau, ptr(un_d), ptr(us), 1e-10, 10) == 4
        st = _abi.Stats()
        s = lib.paris_viscous_solve_mg(p, 0, ptr(nu_d), tau, ptr(un_d), ptr(us), 1e-14, 1, ct.byref(st))
        assert s == 3 and st.iters == 1 and st.converged == 0


@pytest.mark.parametrize("multigrid", [False, True], ids=["jacobi", "mg"])
def test_viscous_fullsize_sampled(paris, multigrid):
    """256^3 drop field in the configuration `bench.py --viscous` times: u* of
    each component at 2048 seeded unknowns against a stored full oracle solve
    (golden/viscous256_drops.json, written by make_viscous256_golden.py from the
    oracle alone).  Bar: the SPD form is a strictly diagonally dominant matrix
    whose rows exceed their off-diagonal sums by 1/(tau nu), so (Varah)
    ||A^-1||_inf <= tau max nu and ||u* - u*_oracle||_inf <= tau max nu
    (||r_gpu||_inf + ||r_oracle||_inf): the GPU's stopping test bounds its
    residual by 1e-10 ||b||_inf, the golden file records the oracle's."""
    path = os.path.join(HERE, "golden", "viscous256_drops.json")
    if not os.path.exists(path):
        pytest.skip("golden/viscous256_drops.json not generated")
    with open(path) as fh:
        gold = json.load(fh)
    pr = pi.config2(n=256)
    assert hashlib.sha256(np.ascontiguousarray(pr.C).tobytes()).hexdigest() == gold["C_sha256"]
    g = pr.grid
    tau = gold["tau"]
    with paris.Context(g) as ctx:
        C = dev(pr.C)
        nus = [ctx.face_viscosity(c, C, gold["mu1"], gold["mu2"], pr.rho1, pr.rho2) for c in range(3)]
        numax = max(float(nu.max()) for nu in nus)
        assert abs(gold["tau_nu_over_h2"] * g.h ** 2 / numax - tau) <= 1e-15 * tau
        for c in range(3):
            un = (pr.u, pr.v, pr.w)[c]
            us, st = ctx.viscous_solve(c, nus[c], tau, dev(un), tol=1e-10, multigrid=multigrid)
            assert st["converged"] == 1 and st["rel_res_l2"] <= 1e-10 and st["rel_res_linf"] <= 1e-10
            x = V.interior(g, c, host(us)).ravel()
            nu = V.interior(g, c, host(nus[c]))
            binf = np.abs(V.interior(g, c, un) / (tau * nu)).max()
            rec = gold["components"][c]
            bound = tau * nu.max() * (1e-10 + rec["rel_res_linf"]) * binf + 1e-14 * rec["x_max_abs"]
            err = np.abs(x[rec["unknowns"]] - np.asarray(rec["x"])).max()
            assert err <= bound, (c, err, bound)
