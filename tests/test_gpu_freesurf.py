"""Free-surface projections on the GPU (through the C ABI), Sec. 3.7.5: the
ghost-fluid projection in the liquid and the phantom projection in two gas
layers, against the oracle (oracle/freesurf.py) element by element, against
the exact linear profile between two free surfaces and the Laplace pressure
of a constant curvature, and against zero divergence afterwards."""
import numpy as np
import pytest

import oracle
import paris_inputs as pi
from oracle import freesurf as FS

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

P, W = pi.PERIODIC, pi.WALL


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


def bubbles(grid, seed, count=3):
    """Gas bubbles (the drops of the seeded generator, read as gas fraction),
    theta ~ U[0.1, 1] on every face, a curvature and a gas pressure per cell,
    u* ~ U[-1, 1]."""
    pr = pi.random_problem(grid, seed=seed, drops=count)
    rng = np.random.default_rng([300, seed])
    theta = [rng.uniform(0.1, 1.0, grid.face_shape(a)) for a in range(3)]
    kappa = rng.normal(0.0, 20.0, grid.shape)
    p_gas = 1.0 + 0.1 * rng.normal(size=grid.shape)
    return pr, theta, kappa, p_gas


GRIDS = [pi.Grid(16, 16, 16, 1 / 16, (P, P, P)), pi.Grid(24, 20, 16, 1 / 24, (P, P, W)),
         pi.Grid(17, 12, 14, 0.05, (W, P, W)), pi.Grid(32, 32, 32, 1 / 32, (P, W, P))]
GID = [f"{g.nx}x{g.ny}x{g.nz}_{''.join('pw'[b] for b in g.bc)}" for g in GRIDS]


@pytest.mark.parametrize("precision", ["FP64", "MIXED"])
@pytest.mark.parametrize("grid", GRIDS, ids=GID)
def test_free_surface_step_matches_oracle(paris, grid, precision):
    """Both forms: the FP64 one, and FP64 refinement around the FP32 V-cycle
    with the diagonal excess in the FP32 operators (without falling back)."""
    pr, theta, kappa, p_gas = bubbles(grid, seed=81)
    rho_l, dt, sigma = 1000.0, 1e-3, 0.07
    want_p, want_u, A, b = FS.gfm_projection(grid, pr.C, rho_l, dt, pr.u, pr.v, pr.w, p_gas, theta, kappa, sigma)
    liq = pr.C < 0.5
    with paris.Context(grid, opts=paris.default_opts(tol=1e-12, precision=getattr(paris, precision))) as ctx:
        u = [dev(x) for x in (pr.u, pr.v, pr.w)]
        p = torch.zeros(grid.shape, dtype=torch.float64, device="cuda")
        st = ctx.free_surface_step(dev(pr.C), rho_l, dt, *u, p, p_gas=dev(p_gas), theta=[dev(t) for t in theta],
                                   kappa=dev(kappa), sigma=sigma)
        assert st["converged"] == 1 and st["rel_res_l2"] <= 1e-12 and st["fell_back"] == 0, st
        ph = host(p)
        scale = np.abs(want_p[liq] - want_p[liq].mean()).max()
        assert np.abs(ph[liq] - want_p[liq]).max() <= 1e-9 * max(scale, 1e-300)
        np.testing.assert_array_equal(ph[~liq], p_gas[~liq])
        umax = max(np.abs(x).max() for x in (pr.u, pr.v, pr.w))
        for a in range(3):
            np.testing.assert_allclose(host(u[a]), want_u[a], rtol=0, atol=1e-9 * umax)
        d = oracle.divergence(grid, *(host(x) for x in u), dt=1.0)
        assert np.abs(d[liq]).max() <= 1e-9 * umax / grid.h


@pytest.mark.parametrize("bc_z", [P, W], ids=["z_periodic", "z_walls"])
def test_linear_profile_between_two_free_surfaces(paris, bc_z):
    """The exact linear pressure through two interface pressures (a liquid
    slab, planes 9..40 of 48, interfaces at theta_lo h and theta_hi h beyond
    the end nodes), u* = 0: p linear to 1e-9 of the pressure difference,
    u = -dt/rho_l times the slope."""
    g = pi.Grid(16, 8, 48, 1 / 48, (P, P, bc_z))
    k_lo, k_hi = 9, 40
    C = np.ones(g.shape)
    C[k_lo:k_hi + 1] = 0.0
    th_lo, th_hi = 0.37, 0.12
    theta = [np.ones(g.face_shape(a)) for a in range(3)]
    theta[2][k_lo] = th_lo
    theta[2][k_hi + 1] = th_hi
    P_lo, P_hi, sigma, rho_l, dt = 2.0, -0.5, 0.05, 500.0, 1e-3
    p_gas = np.where(np.arange(g.nz)[:, None, None] < k_lo, P_lo, P_hi) * np.ones(g.shape)
    kappa = np.where(C < 0.5, 3.0, 7.0)
    ps_lo, ps_hi = P_lo + sigma * 5.0, P_hi + sigma * 5.0
    z = (np.arange(g.nz) + 0.5) * g.h
    z_lo, z_hi = z[k_lo] - th_lo * g.h, z[k_hi] + th_hi * g.h
    slope = (ps_hi - ps_lo) / (z_hi - z_lo)
    want = ps_lo + slope * (z - z_lo)
    with paris.Context(g, opts=paris.default_opts(tol=1e-13)) as ctx:
        u = [torch.zeros(g.face_shape(a), dtype=torch.float64, device="cuda") for a in range(3)]
        p = torch.zeros(g.shape, dtype=torch.float64, device="cuda")
        st = ctx.free_surface_step(dev(C), rho_l, dt, *u, p, p_gas=dev(p_gas), theta=[dev(t) for t in theta],
                                   kappa=dev(kappa), sigma=sigma)
        assert st["converged"] == 1, st
        ph = host(p)
        for k in range(k_lo, k_hi + 1):
            assert np.abs(ph[k] - want[k]).max() <= 1e-9 * abs(ps_lo - ps_hi)
        uz = host(u[2])
        for k in range(k_lo, k_hi + 2):
            np.testing.assert_allclose(uz[k], -dt / rho_l * slope, rtol=1e-8)


def test_constant_curvature_gives_the_laplace_pressure(paris):
    """One gas pressure and a constant curvature, u* = 0, any theta: p =
    p_gas + sigma kappa in the liquid, u = 0."""
    g = pi.Grid(32, 24, 40, 1 / 32, (W, P, P))
    pr, theta, _, _ = bubbles(g, seed=83, count=5)
    with paris.Context(g) as ctx:
        u = [torch.zeros(g.face_shape(a), dtype=torch.float64, device="cuda") for a in range(3)]
        p = torch.zeros(g.shape, dtype=torch.float64, device="cuda")
        st = ctx.free_surface_step(dev(pr.C), 1000.0, 1e-3, *u, p, p_gas=dev(np.full(g.shape, 1.5)),
                                   theta=[dev(t) for t in theta], kappa=dev(np.full(g.shape, -25.0)), sigma=0.07)
        assert st["converged"] == 1, st
        liq = pr.C < 0.5
        np.testing.assert_allclose(host(p)[liq], 1.5 - 0.07 * 25.0, rtol=1e-9)
        for a in range(3):
            assert np.abs(host(u[a])).max() <= 1e-12


@pytest.mark.parametrize("precision", ["FP64", "MIXED"])
def test_free_surface_at_128(paris, precision):
    """A 128^3 box with 12 bubbles (seven multigrid levels with the diagonal
    excess, dense coarsest solve): converged to 1e-10, zero divergence in the
    liquid, gas-gas faces untouched."""
    g = pi.Grid(128, 128, 128, 1 / 128, (P, P, W))
    pr, theta, kappa, p_gas = bubbles(g, seed=85, count=12)
    liq = pr.C < 0.5
    with paris.Context(g, opts=paris.default_opts(precision=getattr(paris, precision))) as ctx:
        u = [dev(x) for x in (pr.u, pr.v, pr.w)]
        p = torch.zeros(g.shape, dtype=torch.float64, device="cuda")
        st = ctx.free_surface_step(dev(pr.C), 1000.0, 1e-3, *u, p, p_gas=dev(p_gas), theta=[dev(t) for t in theta],
                                   kappa=dev(kappa), sigma=0.07)
        assert st["converged"] == 1 and st["iters"] <= 60 and st["fell_back"] == 0, st
        us = [host(x) for x in u]
    d = oracle.divergence(g, *us, dt=1.0)
    assert np.abs(d[liq]).max() <= 1e-8 / g.h
    gasgas = (~liq) & np.roll(~liq, 1, axis=2)
    np.testing.assert_array_equal(us[0][gasgas], pr.u[gasgas])


@pytest.mark.parametrize("grid", [pi.Grid(20, 18, 16, 0.05, (P, P, P)), pi.Grid(24, 16, 20, 1 / 24, (W, P, W))],
                         ids=["ppp", "wpw"])
def test_phantom_projection_matches_oracle(paris, grid):
    rng = np.random.default_rng(87)
    C = np.zeros(grid.shape)
    C[3:12, 2:11, 4:16] = 1.0  # a gas pocket wider than four cells
    us = [rng.uniform(-1, 1, grid.face_shape(a)) for a in range(3)]
    pi.zero_wall_faces(grid, *us)
    want_P, want_u, cls = FS.phantom_projection(grid, C, *us)
    with paris.Context(grid, opts=paris.default_opts(tol=1e-12)) as ctx:
        u = [dev(x) for x in us]
        Ph, st = ctx.phantom_projection(dev(C), *u)
        assert st["converged"] == 1, st
        np.testing.assert_allclose(host(Ph), want_P, rtol=0, atol=1e-9 * np.abs(want_P).max())
        for a in range(3):
            np.testing.assert_allclose(host(u[a]), want_u[a], rtol=0, atol=1e-9)
        d = oracle.divergence(grid, *(host(x) for x in u), dt=1.0)
        assert np.abs(d[cls == 1]).max() <= 1e-9 / grid.h


def test_free_surface_rejects_invalid_arguments(paris):
    g = pi.Grid(8, 8, 8, 1 / 8)
    with paris.Context(g) as ctx:
        C = torch.zeros(g.shape, dtype=torch.float64, device="cuda")
        u = [torch.zeros(g.face_shape(a), dtype=torch.float64, device="cuda") for a in range(3)]
        p = torch.zeros(g.shape, dtype=torch.float64, device="cuda")
        for rho_l, dt in ((0.0, 1e-3), (1.0, -1.0), (float("nan"), 1e-3)):
            with pytest.raises(paris.ParisError):
                ctx.free_surface_step(C, rho_l, dt, *u, p)
        lib, ptr = ctx.lib, ctx._ptr
        import ctypes as ct
        th = ct.c_void_p(u[0].data_ptr())
        none = ct.c_void_p(None)
        s = lib.paris_free_surface_step(ptr, ct.c_void_p(C.data_ptr()), 1.0, 1e-3, th, none, none, none, 0.0, none,
                                        *(ct.c_void_p(x.data_ptr()) for x in u), ct.c_void_p(p.data_ptr()), None)
        assert s != 0  # one theta array without the other two
        solid = torch.ones(g.shape, dtype=torch.uint8, device="cuda")
        ctx.set_solid(solid)
        with pytest.raises(paris.ParisError):
            ctx.free_surface_step(C, 1.0, 1e-3, *u, p)
        with pytest.raises(paris.ParisError):
            ctx.phantom_projection(C, *u)
        ctx.set_solid(None)
