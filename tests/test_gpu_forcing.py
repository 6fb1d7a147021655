"""Predictor forcing on the GPU (through the C ABI): the capillary CSF term of
Eq. csf2 and gravity as they enter Eq. nonconspredictedvel, fused into the
face-coefficient pass.  Checked element by element against the oracle
(oracle/forcing.py), against the hand-computed face values of the oracle's
own pin, and against the exact balances the projection must keep: a drop
with constant curvature (Laplace pressure, u = 0) and fluid layers at rest
(hydrostatic pressure, u = 0)."""
import numpy as np
import pytest

import oracle
import paris_inputs as pi
from oracle import forcing as F

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


GRIDS = [pi.Grid(32, 32, 32, 1 / 32, (P, P, P)), pi.Grid(24, 20, 16, 1 / 24, (P, P, W)),
         pi.Grid(17, 9, 12, 0.05, (W, P, W)), pi.Grid(6, 5, 3, 0.2, (W, W, W)),
         pi.Grid(2, 2, 2, 0.5, (P, P, P)), pi.Grid(40, 2, 35, 1 / 40, (P, W, P))]
GID = [f"{g.nx}x{g.ny}x{g.nz}_{''.join('pw'[b] for b in g.bc)}" for g in GRIDS]


@pytest.mark.parametrize("with_kappa", [True, False], ids=["kappa", "no_kappa"])
@pytest.mark.parametrize("grid", GRIDS, ids=GID)
def test_predictor_forcing_matches_oracle(paris, grid, with_kappa):
    pr = pi.random_problem(grid, seed=61, rho1=1000.0, rho2=1.2)
    kappa = 40.0 * pi.random_field(grid.shape, seed=62, mean_free=False) if with_kappa else None
    sigma, g, tau = 0.07, (0.3, -1.1, -9.81), 2e-3
    un = [x.copy() for x in (pr.u, pr.v, pr.w)]
    want = F.predictor(grid, *un, pr.C, 0.0 if kappa is None else kappa, sigma, g, pr.rho1, pr.rho2, tau)
    beta_ref = oracle.face_coeffs(grid, pr.C, pr.rho1, pr.rho2)
    with paris.Context(grid) as ctx:
        u = [dev(x) for x in un]
        beta = ctx.predictor_forcing(dev(pr.C), None if kappa is None else dev(kappa), pr.rho1, pr.rho2,
                                     sigma, g, tau, *u)
        for a in range(3):
            np.testing.assert_allclose(host(beta[a]), beta_ref[a], rtol=4e-16, atol=0)
            scale = max(np.abs(want[a]).max(), np.abs(un[a]).max(), 1e-300)
            np.testing.assert_allclose(host(u[a]), want[a], rtol=0, atol=2e-15 * scale)
            if grid.bc[a] == W:  # wall faces are zero whatever u^n held there
                sl = [slice(None)] * 3
                for end in (0, -1):
                    sl[2 - a] = end
                    assert np.all(host(u[a])[tuple(sl)] == 0.0)


def test_hand_computed_face_values(paris):
    """The 2x2x2 case computed by hand in the oracle's pin (sigma 1/2, rho 3/1,
    g = (0.1, 0.2, -0.3), walls in z): with u^n = 0 and tau = 1, u* = a."""
    grid = pi.Grid(2, 2, 2, 0.5, (P, P, W))
    C = np.zeros((2, 2, 2))
    C[0, 0, 0], C[0, 0, 1] = 0.25, 0.75
    kappa = np.full((2, 2, 2), 2.0)
    kappa[0, 0, 1] = 4.0
    with paris.Context(grid) as ctx:
        u = [torch.zeros(grid.face_shape(a), dtype=torch.float64, device="cuda") for a in range(3)]
        ctx.predictor_forcing(dev(C), dev(kappa), 3.0, 1.0, 0.5, (0.1, 0.2, -0.3), 1.0, *u)
        ax, ay, az = (host(x) for x in u)
    np.testing.assert_allclose(ax[0, 0, 1], -0.65, rtol=1e-15)
    np.testing.assert_allclose(ax[0, 0, 0], 0.85, rtol=1e-15)
    np.testing.assert_allclose(ax[1, 0, 1], 0.1, rtol=1e-15)
    np.testing.assert_allclose(ay[0, 0, 0], -0.2, rtol=1e-14)
    np.testing.assert_allclose(ay[0, 1, 0], 0.6, rtol=1e-15)
    np.testing.assert_allclose(az[1, 0, 0], 0.1, rtol=1e-14)
    np.testing.assert_allclose(az[1, 0, 1], 9.0 / 7.0 - 0.3, rtol=1e-15)
    assert np.all(az[0] == 0.0) and np.all(az[2] == 0.0)


@pytest.mark.parametrize("precision", ["FP64", "MIXED"])
@pytest.mark.parametrize("kappa", [-8.0, 3.0])
@pytest.mark.parametrize("grid", [pi.Grid(32, 32, 32, 1 / 32), pi.Grid(32, 32, 32, 1 / 32, (P, P, W)),
                                  pi.Grid(48, 32, 40, 1 / 48, (W, P, W))], ids=["ppp", "ppw", "wpw"])
def test_constant_curvature_is_well_balanced(paris, grid, kappa, precision):
    """Drops at ratio 1000 with a constant kappa, fluid at rest: the forced
    projection step returns u = 0 (to 1e-8 of the capillary u*) and
    p = -sigma kappa (C - mean C), the Laplace jump."""
    pr = pi.random_problem(grid, seed=63, rho1=1000.0, rho2=1.0)
    sigma, dt = 0.07, 1e-3
    zero = [np.zeros(grid.face_shape(a)) for a in range(3)]
    ustar = F.predictor(grid, *zero, pr.C, kappa, sigma, (0.0, 0.0, 0.0), pr.rho1, pr.rho2, dt)
    smax = max(np.abs(x).max() for x in ustar)
    with paris.Context(grid, opts=paris.default_opts(precision=getattr(paris, precision))) as ctx:
        u = [dev(x) for x in zero]
        p = torch.zeros(grid.shape, dtype=torch.float64, device="cuda")
        st = ctx.projection_step_forced(dev(pr.C), dev(np.full(grid.shape, kappa)), pr.rho1, pr.rho2, sigma,
                                        (0.0, 0.0, 0.0), dt, *u, p)
        assert st["converged"] == 1, st
        for a in range(3):
            assert np.abs(host(u[a])).max() <= 1e-8 * smax
        pe = -sigma * kappa * (pr.C - pr.C.mean())
        assert np.abs(host(p) - pe).max() <= 1e-8 * np.abs(pe).max()


@pytest.mark.parametrize("precision", ["FP64", "MIXED"])
@pytest.mark.parametrize("grid", [pi.Grid(16, 16, 64, 1 / 16, (P, P, W)), pi.Grid(32, 32, 128, 1 / 32, (P, P, W))],
                         ids=["16x16x64", "32x32x128"])
def test_layers_at_rest_stay_at_rest(paris, grid, precision):
    """Heavy fluid under light, walls in z, gravity only, from rest: u = 0 and
    p_{k+1} - p_k = g h rho_f (the discrete hydrostatic balance)."""
    pr = pi.layered_problem(grid)
    g = (0.0, 0.0, pr.extra["g_z"])
    with paris.Context(grid, opts=paris.default_opts(precision=getattr(paris, precision))) as ctx:
        u = [torch.zeros(grid.face_shape(a), dtype=torch.float64, device="cuda") for a in range(3)]
        p = torch.zeros(grid.shape, dtype=torch.float64, device="cuda")
        st = ctx.projection_step_forced(dev(pr.C), None, pr.rho1, pr.rho2, 0.0, g, pr.dt, *u, p)
        assert st["converged"] == 1, st
        for a in range(3):
            assert np.abs(host(u[a])).max() <= 1e-8 * abs(pr.dt * g[2])
    rho = pr.rho2 + (pr.rho1 - pr.rho2) * pr.C[:, 0, 0]
    dp = g[2] * grid.h * 0.5 * (rho[1:] + rho[:-1])
    pz = np.concatenate([[0.0], np.cumsum(dp)])
    pe = np.broadcast_to(pz[:, None, None], grid.shape) - pz.mean()
    assert np.abs(host(p) - pe).max() <= 1e-8 * np.abs(pe).max()


@pytest.mark.parametrize("precision", ["FP64", "MIXED"])
@pytest.mark.parametrize("grid", [pi.Grid(32, 32, 32, 1 / 32, (P, P, W)), pi.Grid(24, 20, 16, 1 / 24, (W, P, P))],
                         ids=["32ppw", "24x20x16wpp"])
def test_forced_projection_step_matches_oracle(paris, grid, precision):
    """A full forced step from a random u^n with a random curvature field and
    gravity: u^{n+1} and p against the oracle's predictor followed by the
    oracle's projection."""
    pr = pi.random_problem(grid, seed=64, rho1=1000.0, rho2=1.2)
    kappa = 30.0 * pi.random_field(grid.shape, seed=65, mean_free=False)
    sigma, g = 0.07, (0.0, -0.5, -9.81)
    un = [x.copy() for x in (pr.u, pr.v, pr.w)]
    ustar = F.predictor(grid, *un, pr.C, kappa, sigma, g, pr.rho1, pr.rho2, pr.dt)
    ref = oracle.projection_step(grid, pr.C, pr.rho1, pr.rho2, pr.dt, *ustar)
    with paris.Context(grid, opts=paris.default_opts(precision=getattr(paris, precision))) as ctx:
        u = [dev(x) for x in un]
        p = torch.zeros(grid.shape, dtype=torch.float64, device="cuda")
        st = ctx.projection_step_forced(dev(pr.C), dev(kappa), pr.rho1, pr.rho2, sigma, g, pr.dt, *u, p)
        assert st["converged"] == 1 and st["fell_back"] == 0, st
        e = np.abs(host(p) - ref.p).max() / np.abs(ref.p).max()
        assert e <= 1e-8, e
        umax = max(np.abs(x).max() for x in ustar)
        for a in range(3):
            np.testing.assert_allclose(host(u[a]), ref.u[a], rtol=0, atol=1e-7 * umax)
        d = oracle.divergence(grid, *(host(x) for x in u), dt=1.0)
        assert np.abs(d).max() <= 1e-9 * umax / grid.h


def test_forcing_rejects_invalid_arguments(paris):
    grid = pi.Grid(8, 8, 8, 1 / 8)
    with paris.Context(grid) as ctx:
        C = torch.zeros(grid.shape, dtype=torch.float64, device="cuda")
        u = [torch.zeros(grid.face_shape(a), dtype=torch.float64, device="cuda") for a in range(3)]
        for sigma, g, tau in ((-1.0, (0, 0, 0), 1e-3), (0.1, (0, float("nan"), 0), 1e-3),
                              (0.1, (0, 0, 0), -1e-3), (float("inf"), (0, 0, 0), 1e-3)):
            with pytest.raises(paris.ParisError):
                ctx.predictor_forcing(C, None, 2.0, 1.0, sigma, g, tau, *u)
