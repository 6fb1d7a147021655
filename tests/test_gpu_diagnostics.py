"""The diagnostic and option calls of the C ABI on the GPU: the maximum
discrete divergence (against the oracle's divergence) and replacing the
options of a live context."""
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


GRIDS = [
    pi.Grid(24, 20, 16, 1 / 24, (P, P, W)),
    pi.Grid(17, 9, 12, 0.05, (W, P, W)),
    pi.Grid(6, 5, 3, 0.2, (W, W, W)),
]


@pytest.mark.parametrize("grid", GRIDS, ids=lambda g: f"{g.nx}x{g.ny}x{g.nz}")
def test_max_divergence_matches_oracle(paris, grid):
    """max |grad^h . u| of u* (before the projection) and of u (after it):
    the first equals the oracle's (Eqs. cont2, incompdisc3) to rounding, the
    second meets the projection's bar max |div u| <= 1e-9 max |u*| / h."""
    pr = pi.random_problem(grid, seed=41)
    ref = np.abs(oracle.divergence(grid, pr.u, pr.v, pr.w, 1.0)).max()
    umax = max(np.abs(x).max() for x in (pr.u, pr.v, pr.w))
    # six face values per cell, summed in either side's order, then scaled by 1/h
    tol = 8 * np.finfo(float).eps * 6 * umax / grid.h
    with paris.Context(grid) as ctx:
        u, v, w = dev(pr.u), dev(pr.v), dev(pr.w)
        got = ctx.max_divergence(u, v, w)
        assert abs(got - ref) <= tol
        p = torch.zeros(grid.shape, dtype=torch.float64, device="cuda")
        st = ctx.projection_step(dev(pr.C), pr.rho1, pr.rho2, pr.dt, u, v, w, p)
        assert st["converged"] == 1
        after = ctx.max_divergence(u, v, w)
    assert after <= 1e-9 * umax / grid.h
    ref_after = np.abs(oracle.divergence(grid, *(x.cpu().numpy() for x in (u, v, w)), 1.0)).max()
    assert abs(after - ref_after) <= tol


def test_set_opts_changes_the_tolerance(paris):
    """A context's tolerance replaced in place: a looser tolerance stops
    earlier and still meets itself; invalid options are rejected and leave
    the context usable."""
    grid = pi.Grid(32, 32, 32, 1 / 32, (P, P, W))
    pr = pi.random_problem(grid, seed=42)
    C = dev(pr.C)

    def step(ctx):
        u, v, w = dev(pr.u), dev(pr.v), dev(pr.w)
        p = torch.zeros(grid.shape, dtype=torch.float64, device="cuda")
        return ctx.projection_step(C, pr.rho1, pr.rho2, pr.dt, u, v, w, p)

    with paris.Context(grid, opts=paris.default_opts(precision=paris.FP64, tol=1e-10)) as ctx:
        tight = step(ctx)
        ctx.set_opts(tol=1e-5)
        loose = step(ctx)
        with pytest.raises(paris.ParisError):
            ctx.set_opts(tol=0.0)
        ctx.set_opts(tol=1e-10)
        again = step(ctx)
    assert tight["converged"] == 1 and loose["converged"] == 1 and again["converged"] == 1
    assert loose["rel_res_l2"] <= 1e-5 and loose["rel_res_linf"] <= 1e-5
    assert loose["iters"] < tight["iters"]
    assert again["iters"] > loose["iters"] and again["rel_res_l2"] <= 1e-10
