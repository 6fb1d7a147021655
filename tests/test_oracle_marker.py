"""Pins of the marker-function oracle (oracle/marker.py: Eq. FrontMarker3 of
Sec. 3.4.2, Lap_h I = D G_f with beta = 1) on the CPU: the exact recovery of
a marker from its own discrete gradient, the periodic closed form by FFT,
and the cancelling of two opposite sheets (the paper's thin-film remark)."""
import numpy as np
import pytest

import oracle
import paris_inputs as pi
from oracle import marker as M

P, W = pi.PERIODIC, pi.WALL


def sphere_marker(grid, r=0.3):
    C = np.zeros(grid.shape)
    L = grid.lengths
    pi.add_sphere(C, grid, (0.5 * L[0], 0.5 * L[1], 0.5 * L[2]), r * min(L))
    return C


@pytest.mark.parametrize("grid", [pi.Grid(16, 16, 16, 1 / 16), pi.Grid(20, 12, 14, 0.05, (W, P, W))],
                         ids=["ppp", "wpw"])
def test_marker_recovered_from_its_discrete_gradient(grid):
    """G = the face gradient of a known marker (a sub-sampled sphere): the
    solve returns that marker exactly (its mean given)."""
    I0 = sphere_marker(grid)
    G = oracle.face_gradient(grid, I0)
    I, res = M.marker_function(grid, *G, I0.mean())
    assert res.rel_res_l2 <= 1e-12
    assert np.abs(I - I0).max() <= 1e-10


def test_periodic_closed_form():
    """Periodic box: Lap_h I = D G solved by FFT with the eigenvalues
    -(4/h^2) sum sin^2(pi k/n) of the 7-point Laplacian."""
    g = pi.Grid(12, 10, 8, 0.1)
    rng = np.random.default_rng(5)
    G = [rng.standard_normal(g.face_shape(a)) for a in range(3)]
    I, _ = M.marker_function(g, *G, 0.25)
    b = oracle.divergence(g, *G, dt=1.0)
    kz, ky, kx = np.meshgrid(*(np.arange(n) for n in g.shape), indexing="ij")
    lam = -(4 / g.h ** 2) * (np.sin(np.pi * kx / g.nx) ** 2 + np.sin(np.pi * ky / g.ny) ** 2 +
                             np.sin(np.pi * kz / g.nz) ** 2)
    bh = np.fft.fftn(b)
    lam[0, 0, 0] = 1.0
    Ih = bh / lam
    Ih[0, 0, 0] = 0.25 * g.ncells
    want = np.real(np.fft.ifftn(Ih))
    assert np.abs(I - want).max() <= 1e-11 * np.abs(want).max()


def test_opposite_sheets_cancel():
    """Two gradient sheets of opposite sign on the same faces (a film too
    thin for the grid) leave no marker: I = its mean everywhere."""
    g = pi.Grid(10, 10, 10, 0.1, (P, P, W))
    G = [np.zeros(g.face_shape(a)) for a in range(3)]
    G[2][5] = 1.0 / g.h
    G[2][5] += -1.0 / g.h
    I, _ = M.marker_function(g, *G, 0.4)
    assert np.all(np.abs(I - 0.4) <= 1e-14)
