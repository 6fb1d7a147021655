"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Bars (from the method's statement): FP64 relative residual <= 1e-10 in the L2
and L-infinity norms, ||p - p_oracle||_inf / ||p_oracle||_inf <= 1e-8 after
mean removal, max|div u| <= 1e-9 max|u*|/h.  Face coefficients, divergence
and the velocity correction are element-wise checks at a few ulp.
"""
import dataclasses

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


def ctx_for(paris, grid, **opts):
    return paris.Context(grid, opts=paris.default_opts(**opts))


GRIDS = [
    pi.Grid(32, 32, 32, 1 / 32, (P, P, P)),
    pi.Grid(24, 20, 16, 1 / 24, (P, P, W)),
    pi.Grid(17, 9, 12, 0.05, (W, P, W)),
    pi.Grid(6, 5, 3, 0.2, (W, W, W)),
    pi.Grid(2, 2, 2, 0.5, (P, P, P)),
    pi.Grid(48, 2, 10, 1 / 48, (P, W, P)),
]
GID = [f"{g.nx}x{g.ny}x{g.nz}_{''.join('pw'[b] for b in g.bc)}" for g in GRIDS]


@pytest.mark.parametrize("grid", GRIDS, ids=GID)
def test_face_coeffs_match_oracle(paris, grid):
    pr = pi.random_problem(grid, seed=1, rho1=1000.0)
    ref = oracle.face_coeffs(grid, pr.C, pr.rho1, pr.rho2)
    with ctx_for(paris, grid) as ctx:
        got = ctx.face_coeffs(dev(pr.C), pr.rho1, pr.rho2)
        for a in range(3):
            np.testing.assert_allclose(host(got[a]), ref[a], rtol=4e-16, atol=0)


@pytest.mark.parametrize("grid", GRIDS, ids=GID)
def test_divergence_matches_oracle(paris, grid):
    pr = pi.random_problem(grid, seed=2)
    ref = oracle.divergence(grid, pr.u, pr.v, pr.w, pr.dt)
    mref = ref.mean()
    with ctx_for(paris, grid) as ctx:
        rhs, mean = ctx.divergence(dev(pr.u), dev(pr.v), dev(pr.w), pr.dt)
        scale = np.abs(ref).max()
        np.testing.assert_allclose(host(rhs), ref - mref, rtol=0, atol=1e-14 * scale)
        assert abs(mean - mref) <= 1e-14 * scale


@pytest.mark.parametrize("grid", GRIDS, ids=GID)
def test_project_matches_oracle(paris, grid):
    pr = pi.random_problem(grid, seed=3, rho1=50.0)
    beta = oracle.face_coeffs(grid, pr.C, pr.rho1, pr.rho2)
    p = pi.random_field(grid.shape, seed=4)
    ref = oracle.project(grid, *beta, p, pr.dt, pr.u, pr.v, pr.w)
    with ctx_for(paris, grid) as ctx:
        u, v, w = dev(pr.u), dev(pr.v), dev(pr.w)
        ctx.project(*(dev(b) for b in beta), dev(p), pr.dt, u, v, w)
        for a, x in enumerate((u, v, w)):
            np.testing.assert_allclose(host(x), ref[a], rtol=0, atol=1e-14 * np.abs(ref[a]).max())


def _check_solution(grid, pr, ref, p_gpu, u_gpu, st, tol=1e-10, perr=1e-8):
    # residual of the GPU pressure under the ORACLE's operator (FP64 CSR)
    b = ref.rhs - ref.rhs.mean()
    r = b - ref.op.apply_L(p_gpu)
    assert np.linalg.norm(r) <= tol * np.linalg.norm(b) * 1.01, (np.linalg.norm(r) / np.linalg.norm(b), st)
    assert np.abs(r).max() <= tol * np.abs(b).max() * 1.01, (np.abs(r).max() / np.abs(b).max(), st)
    assert abs(p_gpu.mean()) <= 1e-12 * np.abs(p_gpu).max()
    e = np.abs(p_gpu - ref.p).max() / np.abs(ref.p).max()
    assert e <= perr, (e, st)
    umax = max(np.abs(x).max() for x in (pr.u, pr.v, pr.w))
    d = oracle.divergence(grid, *u_gpu, dt=1.0)
    assert np.abs(d).max() <= 1e-9 * umax / grid.h
    for a in range(3):
        np.testing.assert_allclose(u_gpu[a], ref.u[a], rtol=0, atol=1e-7 * umax)


@pytest.mark.parametrize("precision", ["FP64", "MIXED"])
@pytest.mark.parametrize("grid", GRIDS, ids=GID)
def test_projection_step_matches_oracle(paris, grid, precision):
    pr = pi.random_problem(grid, seed=5, rho1=1000.0)
    ref = oracle.projection_step(grid, pr.C, pr.rho1, pr.rho2, pr.dt, pr.u, pr.v, pr.w)
    with ctx_for(paris, grid, precision=getattr(paris, precision)) as ctx:
        u, v, w = dev(pr.u), dev(pr.v), dev(pr.w)
        p = torch.zeros(grid.shape, dtype=torch.float64, device="cuda")
        st = ctx.projection_step(dev(pr.C), pr.rho1, pr.rho2, pr.dt, u, v, w, p)
        assert st["converged"] == 1 and st["fell_back"] == 0, st
        _check_solution(grid, pr, ref, host(p), (host(u), host(v), host(w)), st)


@pytest.mark.parametrize("precision", ["FP64", "MIXED"])
def test_config1_drop32(paris, precision):
    """The 32^3 drop (rho 10/1, u* from seed 0): full parity."""
    pr = pi.config1()
    g = pr.grid
    ref = oracle.projection_step(g, pr.C, pr.rho1, pr.rho2, pr.dt, pr.u, pr.v, pr.w)
    with ctx_for(paris, g, precision=getattr(paris, precision)) as ctx:
        u, v, w = dev(pr.u), dev(pr.v), dev(pr.w)
        p = torch.zeros(g.shape, dtype=torch.float64, device="cuda")
        st = ctx.projection_step(dev(pr.C), pr.rho1, pr.rho2, pr.dt, u, v, w, p)
        _check_solution(g, pr, ref, host(p), (host(u), host(v), host(w)), st)


@pytest.mark.parametrize("precision", ["FP64", "MIXED"])
def test_drops_walls_64(paris, precision):
    """The 256^3 drop-field recipe at 64^3: walls in z, ratio 1000, 64 drops."""
    pr = pi.config2(n=64)
    g = pr.grid
    ref = oracle.projection_step(g, pr.C, pr.rho1, pr.rho2, pr.dt, pr.u, pr.v, pr.w)
    with ctx_for(paris, g, precision=getattr(paris, precision)) as ctx:
        u, v, w = dev(pr.u), dev(pr.v), dev(pr.w)
        p = torch.zeros(g.shape, dtype=torch.float64, device="cuda")
        st = ctx.projection_step(dev(pr.C), pr.rho1, pr.rho2, pr.dt, u, v, w, p)
        assert st["iters"] <= 30, st
        _check_solution(g, pr, ref, host(p), (host(u), host(v), host(w)), st)


LAYERED = [pi.Grid(16, 16, 64, 1 / 16, (P, P, W)), pi.Grid(32, 32, 128, 1 / 32, (P, P, W))]


@pytest.mark.parametrize("noise", [0.0, 0.1], ids=["hydrostatic", "noisy"])
@pytest.mark.parametrize("precision", ["FP64", "MIXED"])
@pytest.mark.parametrize("grid", LAYERED, ids=lambda g: f"{g.nx}x{g.ny}x{g.nz}")
def test_layered_density_walls_z(paris, grid, precision, noise):
    """Heavy fluid (1000) under light (1.2) below a flat interface, walls in
    z, u* = dt g on the z-faces (plus noise): the constant null-space part of
    the residual has to stay out of the solve here (Eq. poisson with Neumann
    walls).  Full parity with the oracle; from rest (no noise) the exact
    discrete answer is hydrostatic, u = 0."""
    pr = pi.layered_problem(grid, noise=noise, seed=11)
    ref = oracle.projection_step(grid, pr.C, pr.rho1, pr.rho2, pr.dt, pr.u, pr.v, pr.w)
    if noise == 0.0:
        # the exact discrete answer: u = 0 needs p_{k+1} - p_k = g h rho_f on
        # every z-face, rho_f the mean of the two cells (Eq. fotm)
        rho = pr.rho2 + (pr.rho1 - pr.rho2) * pr.C[:, 0, 0]
        dp = pr.extra["g_z"] * grid.h * 0.5 * (rho[1:] + rho[:-1])
        pz = np.concatenate([[0.0], np.cumsum(dp)])
        pe = np.broadcast_to(pz[:, None, None], grid.shape).copy()
        ref = dataclasses.replace(ref, p=pe - pe.mean(), u=tuple(np.zeros_like(x) for x in ref.u))
    with ctx_for(paris, grid, precision=getattr(paris, precision)) as ctx:
        u, v, w = dev(pr.u), dev(pr.v), dev(pr.w)
        p = torch.zeros(grid.shape, dtype=torch.float64, device="cuda")
        st = ctx.projection_step(dev(pr.C), pr.rho1, pr.rho2, pr.dt, u, v, w, p)
        assert st["converged"] == 1 and st["fell_back"] == 0, st
        ug = (host(u), host(v), host(w))
        _check_solution(grid, pr, ref, host(p), ug, st)
        if noise == 0.0:
            umax = max(np.abs(x).max() for x in (pr.u, pr.v, pr.w))
            assert max(np.abs(x).max() for x in ug) <= 1e-8 * umax


# every smoothed multigrid level has even periodic axes (walls may be odd)
EVEN_GRIDS = [GRIDS[0], pi.Grid(64, 32, 16, 1 / 64, (P, P, W)), pi.Grid(24, 24, 24, 1 / 24),
              pi.Grid(20, 12, 8, 0.05, (W, W, P)), pi.Grid(13, 7, 9, 0.1, (W, W, W)),
              # tall grids: the two-pass sweep runs slab by slab (periodic and wall z)
              pi.Grid(16, 24, 80, 1 / 16), pi.Grid(24, 16, 72, 1 / 24, (P, W, W))]


@pytest.mark.parametrize("precision", ["FP64", "MIXED"])
@pytest.mark.parametrize("grid", EVEN_GRIDS, ids=lambda g: f"{g.nx}x{g.ny}x{g.nz}")
def test_fused_smoother_bit_identical_to_two_pass(paris, grid, precision):
    """The fused red-black sweep does the same arithmetic in the same order as
    two in-place colour passes: the whole solve is bit-identical (periodic
    axes of even length on every smoothed level, where red-black is a true
    two-colouring)."""
    pr = pi.random_problem(grid, seed=8, rho1=1000.0)
    beta = oracle.face_coeffs(grid, pr.C, pr.rho1, pr.rho2)
    b = oracle.divergence(grid, pr.u, pr.v, pr.w, pr.dt)
    out = []
    for sm, slab in ((paris.SMOOTH_RBGS, 0), (paris.SMOOTH_RBGS_2PASS, 0), (paris.SMOOTH_RBGS_2PASS, 16)):
        with ctx_for(paris, grid, precision=getattr(paris, precision), smoother=sm, slab_planes=slab,
                     half_coefficients=0) as ctx:
            p = torch.zeros(grid.shape, dtype=torch.float64, device="cuda")
            st = ctx.poisson_solve(*(dev(x) for x in beta), dev(b), p)
            out.append((host(p), st["iters"]))
    for q in (1, 2):
        assert out[0][1] == out[q][1]
        np.testing.assert_array_equal(out[0][0], out[q][0])


TAIL_GRIDS = [pi.Grid(128, 128, 128, 1 / 128, (P, P, W)), pi.Grid(96, 64, 48, 1 / 96, (W, P, W)),
              pi.Grid(64, 64, 64, 1 / 64, (W, W, W)), pi.Grid(160, 40, 40, 1 / 160, (P, W, W))]


@pytest.mark.parametrize("precision", ["FP64", "MIXED"])
@pytest.mark.parametrize("grid", TAIL_GRIDS, ids=lambda g: f"{g.nx}x{g.ny}x{g.nz}_{''.join('pw'[b] for b in g.bc)}")
def test_coarse_tail_bit_identical(paris, grid, precision):
    """The small levels of the V-cycle as one launch per step and level, and
    in one single-block launch: the same arithmetic in the same order, so the
    projection step's p and u are identical bit for bit (full coarsening and
    semi-coarsening, walls and periodic axes; the
    periodic axes have even length on every smoothed level, where red-black
    is a true two-colouring and the order of the updates within a colour
    pass does not matter)."""
    pr = pi.random_problem(grid, seed=12, rho1=1000.0)
    out = []
    for tail in (0, 1):
        with ctx_for(paris, grid, precision=getattr(paris, precision), coarse_tail=tail) as ctx:
            u = [dev(x) for x in (pr.u, pr.v, pr.w)]
            p = torch.zeros(grid.shape, dtype=torch.float64, device="cuda")
            st = ctx.projection_step(dev(pr.C), pr.rho1, pr.rho2, pr.dt, *u, p)
            assert st["converged"] == 1, (tail, st)
            out.append((host(p), [host(x) for x in u], st["iters"]))
    assert out[1][2] == out[0][2]
    np.testing.assert_array_equal(out[1][0], out[0][0])
    for a in range(3):
        np.testing.assert_array_equal(out[1][1][a], out[0][1][a])


@pytest.mark.parametrize("precision", ["FP64", "MIXED"])
@pytest.mark.parametrize("grid", GRIDS[:4], ids=GID[:4])
def test_jacobi_smoother_matches_oracle(paris, grid, precision):
    """The paper's GPU iteration (damped Jacobi) as the V-cycle smoother."""
    pr = pi.random_problem(grid, seed=9, rho1=100.0)
    ref = oracle.projection_step(grid, pr.C, pr.rho1, pr.rho2, pr.dt, pr.u, pr.v, pr.w)
    with ctx_for(paris, grid, precision=getattr(paris, precision), smoother=paris.SMOOTH_JACOBI,
                 omega=0.8, max_iter=400) as ctx:
        u, v, w = dev(pr.u), dev(pr.v), dev(pr.w)
        p = torch.zeros(grid.shape, dtype=torch.float64, device="cuda")
        st = ctx.projection_step(dev(pr.C), pr.rho1, pr.rho2, pr.dt, u, v, w, p)
        _check_solution(grid, pr, ref, host(p), (host(u), host(v), host(w)), st)


@pytest.mark.parametrize("rho1,rho2", [(1000.0, 1.0), (1e-3, 7.5), (3.3e4, 2.2e-2), (1.0, 1.0)])
def test_face_coefficient_reciprocal_within_four_ulp(paris, rho1, rho2):
    """beta = 2/(rho_L + rho_R) is computed by Newton-Raphson on the GPU (within
    one ulp of the correctly rounded quotient).  The GPU forms rho/2 =
    (rho1/2) C + (rho2/2)(1 - C) with one fused multiply-add where the oracle
    rounds rho1 C + rho2 (1 - C) three times, so the two rho differ by up to
    ~2 ulp each; the bound checked over random mixtures is therefore 4 ulp."""
    grid = pi.Grid(64, 32, 16, 1 / 64, (P, W, P))
    C = np.random.default_rng(5).uniform(0.0, 1.0, size=grid.shape)
    ref = oracle.face_coeffs(grid, C, rho1, rho2)
    with ctx_for(paris, grid) as ctx:
        got = ctx.face_coeffs(dev(C), rho1, rho2)
        for a in range(3):
            g, r = host(got[a]), ref[a]
            nz = r != 0
            assert np.all(g[~nz] == 0)
            ulps = np.abs(g[nz] - r[nz]) / np.spacing(np.abs(r[nz]))
            assert ulps.max() <= 4.0, ulps.max()


def test_unaligned_pressure_buffer(paris):
    """p may start at any 8-byte boundary (a view into a larger buffer): the
    vectorised kernels fall back to scalar accesses."""
    grid = pi.Grid(24, 20, 16, 1 / 24, (P, P, W))
    pr = pi.random_problem(grid, seed=12, rho1=100.0)
    ref = oracle.projection_step(grid, pr.C, pr.rho1, pr.rho2, pr.dt, pr.u, pr.v, pr.w)
    for prec in ("FP64", "MIXED"):
        with ctx_for(paris, grid, precision=getattr(paris, prec)) as ctx:
            u, v, w = dev(pr.u), dev(pr.v), dev(pr.w)
            buf = torch.zeros(grid.ncells + 1, dtype=torch.float64, device="cuda")
            p = buf[1:].view(grid.shape)
            assert p.data_ptr() % 16 == 8
            st = ctx.projection_step(dev(pr.C), pr.rho1, pr.rho2, pr.dt, u, v, w, p)
            _check_solution(grid, pr, ref, host(p), (host(u), host(v), host(w)), st)


@pytest.mark.parametrize("half", [0, 1])
def test_mixed_with_and_without_fp16_coefficients(paris, half):
    """FP16 copies of beta in the finest-level V-cycle passes change the
    preconditioner only: the solve still meets every bar."""
    pr = pi.config2(n=64)
    g = pr.grid
    ref = oracle.projection_step(g, pr.C, pr.rho1, pr.rho2, pr.dt, pr.u, pr.v, pr.w)
    with ctx_for(paris, g, precision=paris.MIXED, half_coefficients=half) as ctx:
        u, v, w = dev(pr.u), dev(pr.v), dev(pr.w)
        p = torch.zeros(g.shape, dtype=torch.float64, device="cuda")
        st = ctx.projection_step(dev(pr.C), pr.rho1, pr.rho2, pr.dt, u, v, w, p)
        assert st["fell_back"] == 0 and st["iters"] <= 30, st
        _check_solution(g, pr, ref, host(p), (host(u), host(v), host(w)), st)


# even grids whose second level halves every axis: the mixed projection step
# rebuilds the finest level's FP32 operator from the volume fraction there
VOF_GRIDS = [pi.Grid(32, 32, 32, 1 / 32), pi.Grid(64, 32, 16, 1 / 64, (P, P, W)),
             pi.Grid(24, 20, 16, 1 / 24, (W, P, W)), pi.Grid(20, 12, 8, 0.05, (W, W, P)),
             pi.Grid(132, 20, 36, 1 / 132, (P, W, P)), pi.Grid(16, 8, 8, 1 / 16, (W, W, W)),
             # nx/2 odd: the finest level runs the plane-walking (ring) kernels
             # instead of the plane-tile ones, which need an even nx/2
             pi.Grid(30, 20, 12, 1 / 30, (P, W, P)), pi.Grid(22, 12, 16, 1 / 22, (W, P, W))]


@pytest.mark.parametrize("vof", [0, 1])
@pytest.mark.parametrize("grid", VOF_GRIDS, ids=lambda g: f"{g.nx}x{g.ny}x{g.nz}_{''.join('pw'[b] for b in g.bc)}")
def test_level0_from_volume_fraction(paris, grid, vof):
    """The mixed projection step with the finest level's FP32 operator read
    from FP32 face arrays (vof=0) or rebuilt from an FP32 copy of C in the
    colour passes, restriction and inner CG product (vof=1): both meet every
    bar.  The profiler's byte counts show which path ran (a vof colour pass
    moves 10-12 bytes per cell, a face-array pass 20-22)."""
    pr = pi.random_problem(grid, seed=21, rho1=1000.0)
    ref = oracle.projection_step(grid, pr.C, pr.rho1, pr.rho2, pr.dt, pr.u, pr.v, pr.w)
    with ctx_for(paris, grid, precision=paris.MIXED, level0_density=vof) as ctx:
        u, v, w = dev(pr.u), dev(pr.v), dev(pr.w)
        p = torch.zeros(grid.shape, dtype=torch.float64, device="cuda")
        ctx.profile(True)
        st = ctx.projection_step(dev(pr.C), pr.rho1, pr.rho2, pr.dt, u, v, w, p)
        prof = ctx.profile_read()["smooth0"]
        ctx.profile(False)
        assert st["converged"] == 1 and st["fell_back"] == 0, st
        per_cell = prof["bytes"] / prof["timed"] / grid.ncells
        assert (per_cell <= 12.01) if vof else (per_cell >= 20.0), per_cell
        _check_solution(grid, pr, ref, host(p), (host(u), host(v), host(w)), st)


@pytest.mark.parametrize("grid", [pi.Grid(16, 24, 80, 1 / 16), pi.Grid(24, 16, 72, 1 / 24, (P, W, W))],
                         ids=["16x24x80_ppp", "24x16x72_pww"])
def test_level0_density_slabs_bit_identical(paris, grid):
    """Slab-ordered colour passes see the same values as whole-grid passes,
    also when the finest level is rebuilt from the volume fraction."""
    pr = pi.random_problem(grid, seed=22, rho1=300.0)
    out = []
    for slab in (0, 16):
        with ctx_for(paris, grid, precision=paris.MIXED, slab_planes=slab) as ctx:
            u, v, w = dev(pr.u), dev(pr.v), dev(pr.w)
            p = torch.zeros(grid.shape, dtype=torch.float64, device="cuda")
            st = ctx.projection_step(dev(pr.C), pr.rho1, pr.rho2, pr.dt, u, v, w, p)
            assert st["converged"] == 1
            out.append((host(p), st["iters"]))
    assert out[0][1] == out[1][1]
    np.testing.assert_array_equal(out[0][0], out[1][0])


@pytest.mark.parametrize("shift", [0, -3, 7, -40, 40])
def test_integer_conversions_and_reciprocal_match_the_gpu(paris, shift):
    """The kernels convert FP64 <-> FP32 (with a power-of-two scaling) by
    integer operations on the IEEE fields and form FP64 reciprocals by
    Newton-Raphson; the self-check compares both with the GPU's conversion
    and division instructions over values spanning the exponent range, exact
    rounding ties and special values."""
    rng = np.random.default_rng(17)
    v = rng.standard_normal(200000) * 10.0 ** rng.integers(-45, 45, 200000)
    # values exactly at and next to the FP32 rounding boundary
    f = rng.standard_normal(20000).astype(np.float32).astype(np.float64)
    bits = f.view(np.uint64)
    ties = np.concatenate([(bits + d).view(np.float64) for d in (0x10000000, 0x0FFFFFFF, 0x10000001, 0x30000000)])
    special = np.array([0.0, -0.0, np.inf, -np.inf, np.nan, 3.4028234663852886e38, 1.1754943508222875e-38, 1e-320])
    x = np.concatenate([v, ties, special, np.abs(v)])
    assert paris.check_arithmetic(dev(x), shift) == 0


@pytest.mark.parametrize("grid", VOF_GRIDS[:4], ids=lambda g: f"{g.nx}x{g.ny}x{g.nz}_{''.join('pw'[b] for b in g.bc)}")
def test_refinement_residual_matches_fp64_residual(paris, grid):
    """With the finest level rebuilt from rho/2 the mixed form updates the
    FP64 residual in double-float arithmetic (r <- r - A d) instead of
    recomputing f - A x; the norms it reports agree with a full FP64 residual
    of the returned p to 2e-12 (relative to the right-hand side)."""
    pr = pi.random_problem(grid, seed=23, rho1=1000.0)
    with ctx_for(paris, grid, precision=paris.MIXED) as ctx:
        u, v, w = dev(pr.u), dev(pr.v), dev(pr.w)
        p = torch.zeros(grid.shape, dtype=torch.float64, device="cuda")
        st = ctx.projection_step(dev(pr.C), pr.rho1, pr.rho2, pr.dt, u, v, w, p)
        assert st["converged"] == 1 and st["fell_back"] == 0 and st["outer_iters"] >= 2, st
        bx, by, bz = ctx.face_coeffs(dev(pr.C), pr.rho1, pr.rho2)
        rhs = torch.empty(grid.shape, dtype=torch.float64, device="cuda")
        ctx.divergence(dev(pr.u), dev(pr.v), dev(pr.w), pr.dt, rhs)
        l2, linf = ctx.residual_norms(bx, by, bz, rhs, p)
        print(f"reported {st['rel_res_l2']:.3e} {st['rel_res_linf']:.3e}  FP64 {l2:.3e} {linf:.3e}")
        assert abs(st["rel_res_l2"] - l2) <= 2e-12 and abs(st["rel_res_linf"] - linf) <= 2e-12
        assert l2 <= 1e-10 and linf <= 1e-10


def test_stream_rates_probe(paris):
    """The streaming probe returns positive rates below any plausible DRAM
    figure for vectors larger than L2, leaves a, b, c untouched, writes
    o = a + b/2, and rejects misaligned or mis-sized arguments."""
    n = 40 * 1024 * 1024  # 160 MB per vector
    g = torch.Generator(device="cuda").manual_seed(5)
    a, b, c = (torch.rand(n, device="cuda", generator=g) for _ in range(3))
    a0, b0, c0 = a.clone(), b.clone(), c.clone()
    o = torch.empty(n, device="cuda")
    rd, tr = paris.stream_rates(a, b, c, o, reps=3)
    assert 100.0 < rd < 20000.0 and 100.0 < tr < 20000.0, (rd, tr)
    assert torch.equal(a, a0) and torch.equal(b, b0) and torch.equal(c, c0)
    assert torch.equal(o, torch.addcmul(a, b, torch.full_like(b, 0.5)))
    with pytest.raises(paris.ParisError):
        paris.stream_rates(a[1:], b[1:], c[1:], o[1:])  # 4-byte offset: not 16-byte aligned
    with pytest.raises(paris.ParisError):
        paris.stream_rates(a[:6], b[:6], c[:6], o[:6])  # not a multiple of 4


@pytest.mark.parametrize("pinned", [True, False])
def test_host_buffer_step_matches_device_step(paris, pinned):
    """paris_projection_step_host (copies on a second stream, overlapped with
    the step) returns exactly what paris_projection_step returns on device
    arrays, for pinned and pageable host buffers, twice in a row (reused
    staging buffers, fresh inputs each call)."""
    grid = pi.Grid(48, 32, 40, 1 / 48, (P, P, W))
    pr = pi.random_problem(grid, seed=31, rho1=1000.0)
    with ctx_for(paris, grid, precision=paris.MIXED) as ctx:
        u, v, w = dev(pr.u), dev(pr.v), dev(pr.w)
        p = torch.zeros(grid.shape, dtype=torch.float64, device="cuda")
        st_d = ctx.projection_step(dev(pr.C), pr.rho1, pr.rho2, pr.dt, u, v, w, p)
        ref = [host(t) for t in (u, v, w, p)]
        for _ in range(2):
            hs = [torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).clone()
                  for a in (pr.C, pr.u, pr.v, pr.w, np.zeros(grid.shape))]
            if pinned:
                hs = [t.pin_memory() for t in hs]
            st_h = ctx.projection_step_host(*hs[:1], pr.rho1, pr.rho2, pr.dt, *hs[1:])
            assert st_h["iters"] == st_d["iters"] and st_h["converged"] == 1
            for got, want in zip(hs[1:], ref):
                np.testing.assert_array_equal(got.numpy(), want)


@pytest.mark.parametrize("grid", [pi.Grid(48, 32, 40, 1 / 48, (P, P, W)), pi.Grid(64, 24, 16, 1 / 64, (W, P, P))],
                         ids=["48x32x40_ppw", "64x24x16_wpp"])
def test_level0_tiles_match_column_kernels(paris, grid):
    """The plane-tile finest-level kernels (two pairs per thread) and the
    z-column kernels (one pair per thread) compute the same operator: the
    mixed projection step takes the same iterations with either and returns
    the same p to the last few bits (the inner product's dot products are
    summed in another order)."""
    pr = pi.random_problem(grid, seed=33, rho1=1000.0)
    out = []
    for tiles in (1, 0):
        with ctx_for(paris, grid, precision=paris.MIXED, level0_tiles=tiles, level0_half_rho=0) as ctx:
            u, v, w = dev(pr.u), dev(pr.v), dev(pr.w)
            p = torch.zeros(grid.shape, dtype=torch.float64, device="cuda")
            ctx.profile(True)
            st = ctx.projection_step(dev(pr.C), pr.rho1, pr.rho2, pr.dt, u, v, w, p)
            prof = ctx.profile_read()["smooth0"]
            ctx.profile(False)
            assert st["converged"] == 1 and st["fell_back"] == 0
            assert prof["bytes"] / prof["timed"] / grid.ncells <= 12.01
            out.append((host(p), st["iters"], st["outer_iters"]))
    assert out[0][1:] == out[1][1:]
    p0, p1 = out
    assert np.max(np.abs(p0[0] - p1[0])) <= 1e-9 * np.max(np.abs(p1[0]))


@pytest.mark.parametrize("grid", [pi.Grid(64, 32, 40, 1 / 64, (P, P, W)), pi.Grid(48, 16, 24, 1 / 48, (W, P, P)),
                                  pi.Grid(128, 64, 96, 1 / 128, (P, P, P)), pi.Grid(256, 48, 20, 1 / 256, (P, W, W))],
                         ids=["64x32x40_ppw", "48x16x24_wpp", "128x64x96_ppp", "256x48x20_pww"])
def test_staged_colour_pass_bit_identical_to_register_tiles(paris, grid):
    """The finest colour pass staged in shared memory by bulk asynchronous
    copies (level0_tiles = 2) performs the same operations in the same order
    as the register plane-tile pass (level0_tiles = 1), and the product and
    restriction are the same kernels in both: the mixed projection step
    returns bitwise the same p and u after the same iterations.  The grids
    cover short and long plane runs per block, runs that cross a tile
    boundary, two x-chunks per row (nx = 256), and walls on every axis."""
    pr = pi.random_problem(grid, seed=35, rho1=1000.0)
    out = []
    for tiles in (2, 1):
        with ctx_for(paris, grid, precision=paris.MIXED, level0_tiles=tiles, level0_half_rho=0) as ctx:
            u, v, w = dev(pr.u), dev(pr.v), dev(pr.w)
            p = torch.zeros(grid.shape, dtype=torch.float64, device="cuda")
            st = ctx.projection_step(dev(pr.C), pr.rho1, pr.rho2, pr.dt, u, v, w, p)
            assert st["converged"] == 1 and st["fell_back"] == 0, (tiles, st)
            out.append((host(p), host(u), host(v), host(w), st["iters"], st["outer_iters"]))
    assert out[0][4:] == out[1][4:]
    for a, b in zip(out[0][:4], out[1][:4]):
        np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("grid", [pi.Grid(64, 64, 64, 1 / 64, (P, P, W)), pi.Grid(96, 48, 40, 1 / 96, (W, P, P))],
                         ids=["64_ppw", "96x48x40_wpp"])
@pytest.mark.parametrize("rho1,rho2", [(1000.0, 1.0), (1.0, 1e-4)], ids=["ratio1000", "rho_below_fp16"])
def test_half_density_v_cycle(paris, grid, rho1, rho2):
    """The V-cycle's finest passes reading rho/2 in FP16 (level0_half_rho)
    change the preconditioner only: the step converges in at most one more
    iteration than with FP32 rho/2 and returns p within 1e-8 of it, both
    within the oracle's bar; densities outside FP16's comfortable range
    (rho/2 below 1e-4 here) keep FP32."""
    pr = pi.random_problem(grid, seed=37, rho1=rho1, rho2=rho2)
    ref = oracle.projection_step(grid, pr.C, pr.rho1, pr.rho2, pr.dt, pr.u, pr.v, pr.w)
    out = []
    for half in (1, 0):
        with ctx_for(paris, grid, precision=paris.MIXED, level0_half_rho=half) as ctx:
            u, v, w = dev(pr.u), dev(pr.v), dev(pr.w)
            p = torch.zeros(grid.shape, dtype=torch.float64, device="cuda")
            ctx.profile(True)
            st = ctx.projection_step(dev(pr.C), pr.rho1, pr.rho2, pr.dt, u, v, w, p)
            prof = ctx.profile_read()["smooth0"]
            ctx.profile(False)
            assert st["converged"] == 1 and st["fell_back"] == 0, (half, st)
            out.append((host(p), st["iters"], prof["bytes"] / prof["timed"] / grid.ncells))
    (ph, ih, bh), (pf, i_f, bf) = out
    assert ih <= i_f + 1, (ih, i_f)
    scale = np.abs(ref.p).max()
    assert np.abs(ph - pf).max() <= 1e-8 * scale
    assert np.abs(ph - ref.p).max() <= 1e-8 * scale
    # the bytes the class counts: 2 B of rho/2 a cell fewer per regular pass in the FP16 mode
    if min(rho1, rho2) >= 2e-4:
        assert bh < bf - 1.0
    else:
        assert bh == bf
