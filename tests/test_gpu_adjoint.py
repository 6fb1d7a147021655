"""Adjoint of the projection on the GPU (through the C ABI and the autograd
Function): element-wise against the oracle adjoint, and against central finite
differences of the GPU forward on the 128^3 tanh drop (rho 100/1) for a loss
L = 1/2 ||u - u_target||^2 with a discretely divergence-free target."""
import numpy as np
import pytest

import oracle
import paris_inputs as pi

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


def tanh_drop(grid, r0=0.3, w=0.1):
    c = [(np.arange(n) + 0.5) / n - 0.5 for n in (grid.nz, grid.ny, grid.nx)]
    r = np.sqrt(c[0][:, None, None] ** 2 + c[1][None, :, None] ** 2 + c[2][None, None, :] ** 2)
    return 0.5 * (1.0 - np.tanh((r - r0) / w))


@pytest.mark.parametrize("precision", ["FP64", "MIXED"])
@pytest.mark.parametrize("grid", [pi.Grid(16, 16, 16, 1 / 16), pi.Grid(12, 10, 8, 1 / 12, (P, W, P))],
                         ids=["16p", "12x10x8_wall_y"])
def test_adjoint_matches_oracle(paris, grid, precision):
    rng = np.random.default_rng(41)
    C = tanh_drop(grid)
    u = [rng.uniform(-1, 1, size=grid.face_shape(a)) for a in range(3)]
    pi.zero_wall_faces(grid, *u)
    t = [rng.uniform(-1, 1, size=grid.face_shape(a)) for a in range(3)]
    rho1, rho2, dt = 20.0, 1.0, 0.01
    ref = oracle.projection_step(grid, C, rho1, rho2, dt, *u, tol=1e-14)
    g = [ref.u[a] - t[a] for a in range(3)]
    rgus, rgb, _, _ = oracle.project_adjoint(grid, ref.op, ref.beta, ref.p, dt, *g, tol=1e-14)
    rgC = oracle.face_coeffs_adjoint(grid, rho1, rho2, ref.beta, rgb)
    with paris.Context(grid, opts=paris.default_opts(precision=getattr(paris, precision), tol=1e-12)) as ctx:
        gus, gb, q, st = ctx.project_adjoint(*(dev(b) for b in ref.beta), dev(ref.p), dt,
                                             *(dev(x) for x in g))
        assert st["converged"] == 1
        gC = ctx.face_coeffs_adjoint(rho1, rho2, *(dev(b) for b in ref.beta), *gb)
        for a in range(3):
            np.testing.assert_allclose(host(gus[a]), rgus[a], rtol=0, atol=1e-8 * np.abs(rgus[a]).max())
            np.testing.assert_allclose(host(gb[a]), rgb[a], rtol=0, atol=1e-8 * np.abs(rgb[a]).max())
        np.testing.assert_allclose(host(gC), rgC, rtol=0, atol=1e-8 * np.abs(rgC).max())


def test_autograd_function_matches_abi(paris):
    grid = pi.Grid(16, 12, 8, 1 / 16, (P, P, W))
    rng = np.random.default_rng(3)
    C = dev(tanh_drop(grid)).requires_grad_(True)
    us = [dev(rng.uniform(-1, 1, size=grid.face_shape(a))) for a in range(3)]
    pi.zero_wall_faces(grid, *us)
    us = [x.requires_grad_(True) for x in us]
    t = [dev(rng.uniform(-1, 1, size=grid.face_shape(a))) for a in range(3)]
    with paris.Context(grid, opts=paris.default_opts(precision=paris.FP64, tol=1e-12)) as ctx:
        u, v, w, p = paris.projection(C, *us, ctx, 50.0, 1.0, 1e-3)
        loss = 0.5 * sum(((x - tt) ** 2).sum() for x, tt in zip((u, v, w), t))
        loss.backward()
        bx, by, bz = ctx.face_coeffs(C.detach(), 50.0, 1.0)
        g = [(x - tt).detach().contiguous() for x, tt in zip((u, v, w), t)]
        gus, gb, _, _ = ctx.project_adjoint(bx, by, bz, p, 1e-3, *g)
        gC = ctx.face_coeffs_adjoint(50.0, 1.0, bx, by, bz, *gb)
        for a in range(3):
            np.testing.assert_allclose(host(us[a].grad), host(gus[a]), rtol=0, atol=1e-12)
        np.testing.assert_allclose(host(C.grad), host(gC), rtol=0, atol=1e-12 * host(gC).__abs__().max())


@pytest.fixture(scope="module")
def adjoint128(paris):
    pr = pi.config5(n=128)
    return pr


def _loss_increment(up, um, t):
    """sum (u+ - u-) * ((u+ + u-)/2 - t) = L(u+) - L(u-) without cancellation."""
    s = 0.0
    for a in range(3):
        s += float(((up[a] - um[a]) * (0.5 * (up[a] + um[a]) - t[a])).sum())
    return s


@pytest.mark.parametrize("precision", ["FP64", "MIXED"])
def test_adjoint_against_finite_differences_128(paris, adjoint128, precision):
    """64 entries of u* and 64 of C among those with |grad| >= 1e-3 max|grad|:
    central differences (FP64 forward solves to 1e-14, warm-started from the
    base pressure) agree with the adjoint to 1e-6 relative.
    u is exactly linear in u*, so a central difference in u* has no truncation
    error at any step; its step is 1e-2, which keeps the rounding noise of the
    loss increment (~1e-16 per face over 6.3M faces, divided by twice the
    step) far below the smallest gradients sampled.  u depends on C
    nonlinearly: a two-point central difference at step 1e-6 is limited by
    that noise (~3e-6 absolute, i.e. 2e-5 relative on the smallest sampled
    entries) and at 1e-4 by its h^2 error; the four-point central difference
    (8 (f1 - f-1) - (f2 - f-2)) / 12h with h = 5e-5 has an h^4 error and 50x
    less noise, and is used for C."""
    pr = adjoint128
    g = pr.grid
    t = [dev(x) for x in pr.extra["target"]]
    C0 = dev(pr.C)
    u0 = [dev(x) for x in (pr.u, pr.v, pr.w)]
    fwd = paris.Context(g, opts=paris.default_opts(precision=paris.FP64, tol=1e-14, max_iter=400))
    adj = paris.Context(g, opts=paris.default_opts(precision=getattr(paris, precision), tol=1e-13,
                                                   max_iter=400))

    def forward(C, u, p0):
        uu = [x.clone() for x in u]
        p = p0.clone()
        fwd.projection_step(C, pr.rho1, pr.rho2, pr.dt, *uu, p, check=False)
        return uu, p

    try:
        ub, pb = forward(C0, u0, torch.zeros(g.shape, dtype=torch.float64, device="cuda"))
        bx, by, bz = adj.face_coeffs(C0, pr.rho1, pr.rho2)
        gin = [(ub[a] - t[a]).contiguous() for a in range(3)]
        gus, gb, _, st = adj.project_adjoint(bx, by, bz, pb, pr.dt, *gin)
        assert st["converged"] == 1, st
        gC = host(adj.face_coeffs_adjoint(pr.rho1, pr.rho2, bx, by, bz, *gb))
        gus = [host(x) for x in gus]
        rng = np.random.default_rng(55)
        eps_u, eps_c = 1e-2, 5e-5
        worst_u = worst_c = 0.0
        # u* entries (component chosen at random per sample)
        flat = np.concatenate([x.ravel() for x in gus])
        big = np.flatnonzero(np.abs(flat) >= 1e-3 * np.abs(flat).max())
        sizes = np.cumsum([0] + [x.size for x in gus])
        for idx in rng.choice(big, size=64, replace=False):
            a = int(np.searchsorted(sizes, idx, side="right") - 1)
            f = idx - sizes[a]
            res = []
            for sgn in (1, -1):
                u = [x.clone() for x in u0]
                u[a].view(-1)[f] += sgn * eps_u
                res.append(forward(C0, u, pb)[0])
            fd = _loss_increment(res[0], res[1], t) / (2 * eps_u)
            ad = flat[idx]
            worst_u = max(worst_u, abs(fd - ad) / abs(ad))
        # C entries
        bigC = np.flatnonzero(np.abs(gC.ravel()) >= 1e-3 * np.abs(gC).max())
        for idx in rng.choice(bigC, size=64, replace=False):
            res = {}
            for m in (1, -1, 2, -2):
                C = C0.clone()
                C.view(-1)[idx] += m * eps_c
                res[m] = forward(C, u0, pb)[0]
            d1 = _loss_increment(res[1], res[-1], t)
            d2 = _loss_increment(res[2], res[-2], t)
            fd = (8.0 * d1 - d2) / (12.0 * eps_c)
            ad = gC.ravel()[idx]
            worst_c = max(worst_c, abs(fd - ad) / abs(ad))
        print(f"adjoint {precision}: worst relative difference to finite differences "
              f"u* {worst_u:.2e}, C {worst_c:.2e}")
        assert worst_u <= 1e-6 and worst_c <= 1e-6, (worst_u, worst_c)
    finally:
        fwd.close()
        adj.close()
