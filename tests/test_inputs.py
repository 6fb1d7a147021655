"""Checks of the seeded input generator (no method arithmetic involved)."""
import math

import numpy as np

import paris_inputs as pi


def test_sphere_volume_and_range():
    g = pi.Grid(32, 32, 32, 1.0 / 32)
    C = np.zeros(g.shape)
    pi.add_sphere(C, g, (0.5, 0.5, 0.5), 0.25)
    assert C.min() >= 0 and C.max() <= 1
    vol = C.sum() * g.h ** 3
    assert abs(vol - 4 / 3 * math.pi * 0.25 ** 3) < 2e-3 * vol
    # symmetric about the centre plane
    np.testing.assert_array_equal(C, C[::-1, :, :])


def test_sphere_wraps_periodically():
    g = pi.Grid(16, 16, 16, 1.0 / 16)
    a = np.zeros(g.shape)
    b = np.zeros(g.shape)
    pi.add_sphere(a, g, (0.02, 0.5, 0.5), 0.2)
    pi.add_sphere(b, g, (0.52, 0.5, 0.5), 0.2)
    # shifting the centre by half the box rolls the field by 8 cells (exact:
    # sub-cell positions differ only by the shift)
    np.testing.assert_allclose(np.roll(a, 8, axis=2), b, atol=1.0 / 64 + 1e-12)
    assert abs(a.sum() - b.sum()) <= 2


def test_reproducible():
    a = pi.config2(n=32, drops=8)
    b = pi.config2(n=32, drops=8)
    for x, y in zip((a.C, a.u, a.v, a.w), (b.C, b.u, b.v, b.w)):
        np.testing.assert_array_equal(x, y)


def test_config2_geometry():
    pr = pi.config2(n=64)
    sph = pr.extra["spheres"]
    assert len(sph) == 64
    h = pr.grid.h
    for i, (c1, r1) in enumerate(sph):
        assert 0.02 <= r1 <= 0.08
        assert r1 + 2 * h <= c1[2] <= 1 - r1 - 2 * h
        for c2, r2 in sph[:i]:
            d = [c1[a] - c2[a] for a in range(3)]
            d[0] -= round(d[0]); d[1] -= round(d[1])
            assert math.sqrt(sum(x * x for x in d)) >= r1 + r2 + 2 * h - 1e-12
    assert np.all(pr.w[0] == 0) and np.all(pr.w[-1] == 0)
    assert pr.w.shape == (65, 64, 64) and pr.u.shape == (64, 64, 64)


def test_edge_potential_curl_is_divergence_free():
    g = pi.Grid(12, 10, 8, 1.0 / 12)
    u, v, w = pi.edge_potential_curl(np.random.default_rng(1), g, 5, 3)
    div = (np.roll(u, -1, 2) - u + np.roll(v, -1, 1) - v + np.roll(w, -1, 0) - w) / g.h
    scale = max(np.abs(u).max(), np.abs(v).max(), np.abs(w).max()) / g.h
    assert np.abs(div).max() < 1e-12 * scale
    assert scale > 1.0


def test_config1_definition():
    pr = pi.config1()
    rng = np.random.default_rng(0)
    np.testing.assert_array_equal(pr.u, rng.uniform(-1, 1, size=(32, 32, 32)))
    assert pr.rho1 == 10.0 and pr.rho2 == 1.0 and pr.dt == 1e-3


def test_config4_sizes():
    probs = pi.config4(count=16)
    for p in probs:
        assert all(n in pi.BATCH_AXES for n in (p.grid.nx, p.grid.ny, p.grid.nz))
        assert 1.0 <= p.rho1 <= 1000.0
        assert 1 <= len(p.extra["spheres"]) <= 8
