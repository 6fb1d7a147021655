"""Front-tracking marker function on the GPU (Sec. 3.4.2, Eq. FrontMarker3:
Lap_h I = D G with beta = 1), through the C ABI, against the oracle
(oracle/marker.py) and against the exact recovery of a marker from its own
discrete gradient."""
import numpy as np
import pytest

import oracle
import paris_inputs as pi
from oracle import marker as M

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


GRIDS = [pi.Grid(32, 32, 32, 1 / 32), pi.Grid(24, 20, 16, 1 / 24, (P, P, W)), pi.Grid(17, 9, 12, 0.05, (W, P, W)),
         pi.Grid(64, 48, 40, 1 / 64, (W, W, W))]
GID = [f"{g.nx}x{g.ny}x{g.nz}_{''.join('pw'[b] for b in g.bc)}" for g in GRIDS]


@pytest.mark.parametrize("precision", ["FP64", "MIXED"])
@pytest.mark.parametrize("grid", GRIDS, ids=GID)
def test_marker_recovered_from_its_gradient(paris, grid, precision):
    """G = face gradient of a sub-sampled sphere marker: I comes back."""
    I0 = np.zeros(grid.shape)
    L = grid.lengths
    pi.add_sphere(I0, grid, (0.45 * L[0], 0.5 * L[1], 0.55 * L[2]), 0.3 * min(L))
    G = oracle.face_gradient(grid, I0)
    with paris.Context(grid, opts=paris.default_opts(precision=getattr(paris, precision), tol=1e-12)) as ctx:
        I, st = ctx.marker_function(*(dev(x) for x in G), I0.mean())
        assert st["converged"] == 1, st
        assert np.abs(host(I) - I0).max() <= 1e-9


@pytest.mark.parametrize("precision", ["FP64", "MIXED"])
@pytest.mark.parametrize("grid", GRIDS[:3], ids=GID[:3])
def test_marker_matches_oracle(paris, grid, precision):
    """A general face field G (not a gradient): I against the oracle."""
    rng = np.random.default_rng(91)
    G = [rng.standard_normal(grid.face_shape(a)) for a in range(3)]
    ref, _ = M.marker_function(grid, *G, 0.3)
    with paris.Context(grid, opts=paris.default_opts(precision=getattr(paris, precision))) as ctx:
        I, st = ctx.marker_function(*(dev(x) for x in G), 0.3)
        assert st["converged"] == 1
        Ig = host(I)
    assert abs(Ig.mean() - 0.3) <= 1e-12
    assert np.abs(Ig - ref).max() <= 1e-8 * np.abs(ref - 0.3).max()


def test_marker_argument_checks(paris):
    grid = pi.Grid(16, 16, 16, 1 / 16)
    G = [torch.zeros(grid.face_shape(a), dtype=torch.float64, device="cuda") for a in range(3)]
    with paris.Context(grid) as ctx:
        with pytest.raises(paris.ParisError):
            ctx.marker_function(*G, float("nan"))
        s = torch.ones(grid.shape, dtype=torch.uint8, device="cuda")
        ctx.set_solid(s)
        with pytest.raises(paris.ParisError):
            ctx.marker_function(*G, 0.5)
