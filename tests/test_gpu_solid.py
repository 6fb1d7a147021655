"""Solid cells on the GPU (Sec. 3.8 "Lego" solids, through the C ABI): the
projection with a solid mask against the solid-cell oracle (oracle/solid.py)
element by element, the slab that equals a wall pair, and the argument
checks."""
import numpy as np
import pytest

import oracle
import paris_inputs as pi
from oracle import solid as S

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


def mask_block(grid):
    fl = np.ones(grid.shape, np.uint8)
    nz, ny, nx = grid.shape
    fl[nz // 4:nz // 2, ny // 3:2 * ny // 3, nx // 4:nx // 2 + 1] = 0
    return fl


def mask_obstacles(grid, seed):
    """A few seeded boxes of solid that leave the fluid connected (each box
    is at most a third of every axis and away from the others)."""
    rng = np.random.default_rng([900, seed])
    fl = np.ones(grid.shape, np.uint8)
    nz, ny, nx = grid.shape
    for q in range(3):
        sz, sy, sx = (max(1, n // 5) for n in (nz, ny, nx))
        z0 = (q * nz) // 3 + rng.integers(0, max(1, nz // 3 - sz))
        y0, x0 = rng.integers(0, ny - sy), rng.integers(0, nx - sx)
        fl[z0:z0 + sz, y0:y0 + sy, x0:x0 + sx] = 0
    return fl


CASES = [(pi.Grid(32, 32, 32, 1 / 32, (P, P, P)), "block"), (pi.Grid(24, 20, 16, 1 / 24, (P, P, W)), "block"),
         (pi.Grid(17, 9, 12, 0.05, (W, P, W)), "obstacles"), (pi.Grid(48, 32, 40, 1 / 48, (P, W, P)), "obstacles"),
         (pi.Grid(64, 64, 64, 1 / 64, (P, P, W)), "obstacles")]
CID = [f"{g.nx}x{g.ny}x{g.nz}_{''.join('pw'[b] for b in g.bc)}_{m}" for g, m in CASES]


@pytest.mark.parametrize("precision", ["FP64", "MIXED"])
@pytest.mark.parametrize("case", CASES, ids=CID)
def test_projection_with_solid_matches_oracle(paris, case, precision):
    grid, kind = case
    fl = mask_block(grid) if kind == "block" else mask_obstacles(grid, grid.nx)
    pr = pi.random_problem(grid, seed=81, rho1=1000.0)
    pref, uref, beta_ref, res, b = S.projection_step_solid(grid, pr.C, pr.rho1, pr.rho2, pr.dt, pr.u, pr.v,
                                                           pr.w, fl)
    with paris.Context(grid, opts=paris.default_opts(precision=getattr(paris, precision))) as ctx:
        s = torch.from_numpy(fl).cuda()
        ctx.set_solid(s)
        beta = ctx.face_coeffs(dev(pr.C), pr.rho1, pr.rho2)
        for a in range(3):
            np.testing.assert_allclose(host(beta[a]), beta_ref[a], rtol=4e-16, atol=0)
        u, v, w = dev(pr.u), dev(pr.v), dev(pr.w)
        p = torch.zeros(grid.shape, dtype=torch.float64, device="cuda")
        st = ctx.projection_step(dev(pr.C), pr.rho1, pr.rho2, pr.dt, u, v, w, p)
        assert st["converged"] == 1 and st["fell_back"] == 0, st
        pg = host(p)
        assert np.all(pg[fl == 0] == 0.0)
        assert abs(pg[fl == 1].mean()) <= 1e-12 * np.abs(pg).max()
        # the residual of the GPU pressure under the oracle's masked operator
        op = oracle.Operator(grid, *beta_ref)
        b0 = oracle.null_project(b, fl)
        r = (b0 - op.apply_L(pg))[fl == 1]
        op.close()
        assert np.linalg.norm(r) <= 1e-10 * np.linalg.norm(b0) * 1.01
        assert np.abs(r).max() <= 1e-10 * np.abs(b0).max() * 1.01
        e = np.abs(pg - pref).max() / np.abs(pref).max()
        assert e <= 1e-8, e
        umax = max(np.abs(x).max() for x in (pr.u, pr.v, pr.w))
        flags = S.face_flags(grid, fl)
        for a, x in enumerate((u, v, w)):
            ug = host(x)
            assert np.all(ug[flags[a] == 0] == 0.0)
            np.testing.assert_allclose(ug, uref[a], rtol=0, atol=1e-7 * umax)
        d = oracle.divergence(grid, host(u), host(v), host(w), dt=1.0)
        assert np.abs(d[fl == 1]).max() <= 1e-9 * umax / grid.h


def test_slab_equals_wall_pair_on_the_gpu(paris):
    """Planes 6-9 of a periodic-z 32x24x40 box solid: the same p and u as the
    walls-in-z box of the other 36 planes (mixed form, both on the GPU)."""
    nz, k_lo, k_hi = 40, 6, 9
    g = pi.Grid(32, 24, nz, 1 / 32)
    pr = pi.random_problem(g, seed=82, rho1=300.0)
    fl = np.ones(g.shape, np.uint8)
    fl[k_lo:k_hi + 1] = 0
    order = [(k_hi + 1 + m) % nz for m in range(nz - (k_hi - k_lo + 1))]
    gw = pi.Grid(32, 24, len(order), 1 / 32, (P, P, W))
    ww = np.zeros(gw.face_shape(2))
    for m in range(1, len(order)):
        ww[m] = pr.w[order[m]]
    outs = []
    for grid, C, uvw, mask in ((g, pr.C, (pr.u, pr.v, pr.w), fl),
                               (gw, pr.C[order], (pr.u[order], pr.v[order], ww), None)):
        with paris.Context(grid, opts=paris.default_opts(precision=paris.MIXED, tol=1e-12)) as ctx:
            if mask is not None:
                s = torch.from_numpy(mask).cuda()
                ctx.set_solid(s)
            u, v, w = (dev(x) for x in uvw)
            p = torch.zeros(grid.shape, dtype=torch.float64, device="cuda")
            st = ctx.projection_step(dev(C), pr.rho1, pr.rho2, pr.dt, u, v, w, p)
            assert st["converged"] == 1
            outs.append((host(p), host(u), host(v), host(w)))
    (p1, u1, v1, w1), (p2, u2, v2, w2) = outs
    assert np.abs(p1[order] - p2).max() <= 1e-8 * np.abs(p2).max()
    assert np.abs(u1[order] - u2).max() <= 1e-8 * np.abs(u2).max()
    assert np.abs(v1[order] - v2).max() <= 1e-8 * np.abs(v2).max()
    for m in range(1, len(order)):
        assert np.abs(w1[order[m]] - w2[m]).max() <= 1e-8 * np.abs(w2).max()


def test_clearing_the_solid_restores_the_plain_projection(paris):
    grid = pi.Grid(32, 32, 32, 1 / 32, (P, P, W))
    pr = pi.random_problem(grid, seed=83)
    ref = oracle.projection_step(grid, pr.C, pr.rho1, pr.rho2, pr.dt, pr.u, pr.v, pr.w)
    with paris.Context(grid) as ctx:
        s = torch.from_numpy(mask_block(grid)).cuda()
        ctx.set_solid(s)
        ctx.set_solid(None)
        u, v, w = dev(pr.u), dev(pr.v), dev(pr.w)
        p = torch.zeros(grid.shape, dtype=torch.float64, device="cuda")
        ctx.projection_step(dev(pr.C), pr.rho1, pr.rho2, pr.dt, u, v, w, p)
        assert np.abs(host(p) - ref.p).max() <= 1e-8 * np.abs(ref.p).max()


def test_solid_argument_checks(paris):
    grid = pi.Grid(16, 16, 16, 1 / 16)
    with paris.Context(grid) as ctx:
        with pytest.raises(paris.ParisError):
            ctx.set_solid(torch.zeros(grid.shape, dtype=torch.uint8, device="cuda"))  # no fluid cell
        s = torch.from_numpy(mask_block(grid)).cuda()
        ctx.set_solid(s)
        beta = ctx.face_coeffs(torch.zeros(grid.shape, dtype=torch.float64, device="cuda"), 2.0, 1.0)
        p = torch.zeros(grid.shape, dtype=torch.float64, device="cuda")
        g = [torch.zeros(grid.face_shape(a), dtype=torch.float64, device="cuda") for a in range(3)]
        with pytest.raises(paris.ParisError):
            ctx.project_adjoint(*beta, p, 1e-3, *g)
