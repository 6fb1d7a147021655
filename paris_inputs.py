"""Seeded synthetic inputs for the one-fluid pressure projection.

This module only *creates* input fields: cell volume fractions C of drops and
jets, predicted face velocities u*, and test-only potentials.  It holds none of
the projection's arithmetic (no face coefficients, no divergence, no solve, no
velocity correction), so both the CPU oracle and the CUDA path can take their
inputs from it without sharing any of the method's code.

Grid conventions (staggered MAC grid, Section 3.1 of the paper):

* cells (i, j, k), numpy arrays in C order with shape (nz, ny, nx): x fastest,
  linear index (k*ny + j)*nx + i;
* cubic spacing h, box length L_m = n_m * h along each axis;
* u is stored on x-faces, v on y-faces, w on z-faces.  Face "i-1/2" of cell i
  is stored at index i.  Along a periodic axis a face array has n entries
  (face n-1/2 is face -1/2); along a wall axis it has n+1 entries, and the
  entries 0 and n are the wall faces, where the normal velocity is zero.

Volume fractions follow the paper's sub-grid initialisation (Section 3.5.3):
every cell is split into n_I^3 sub-cells (n_I = 4 here), the sub-cell centre is
classified inside the liquid when the implicit function phi < 0 (a tie phi = 0
counts as outside) and C is the inside count divided by n_I^3.

Random streams use numpy's PCG64: ``default_rng([cfg_id, stream])`` with stream
0 = geometry, 1 = u*, 2 = noise, 3 = targets.  Configuration 1 draws u* from
``default_rng(0)`` as its definition states.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

PERIODIC = 0
WALL = 1

N_SUB = 4  # sub-cells per axis for the volume-fraction initialisation


@dataclass
class Grid:
    nx: int
    ny: int
    nz: int
    h: float
    bc: tuple = (PERIODIC, PERIODIC, PERIODIC)  # per axis (x, y, z)

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)

    @property
    def ncells(self):
        return self.nx * self.ny * self.nz

    def face_shape(self, axis: int):
        """numpy shape (z, y, x) of the face array normal to ``axis`` (0=x, 1=y, 2=z)."""
        n = [self.nz, self.ny, self.nx]
        n[2 - axis] += 1 if self.bc[axis] == WALL else 0
        return tuple(n)

    @property
    def lengths(self):
        return (self.nx * self.h, self.ny * self.h, self.nz * self.h)


@dataclass
class Problem:
    """One projection problem: grid, volume fraction, densities, u*, time step."""
    name: str
    grid: Grid
    C: np.ndarray
    u: np.ndarray
    v: np.ndarray
    w: np.ndarray
    rho1: float
    rho2: float
    dt: float
    tol: float = 1e-10
    extra: dict = field(default_factory=dict)


def _rng(cfg_id: int, stream: int) -> np.random.Generator:
    return np.random.default_rng([cfg_id, stream])


# ---------------------------------------------------------------- geometry ---

def _sub_offsets(h: float) -> np.ndarray:
    """Offsets (s + 1/2)/n_I * h of the sub-cell centres inside a cell."""
    return (np.arange(N_SUB, dtype=np.float64) + 0.5) / N_SUB * h


def _axis_sq(lo: int, hi: int, h: float, centre: float) -> np.ndarray:
    """Squared distances along one axis for cells lo..hi-1 (unwrapped indices):
    array of shape (hi-lo, N_SUB) of (x_sub - centre)^2."""
    i = np.arange(lo, hi, dtype=np.float64)
    x = i[:, None] * h + _sub_offsets(h)[None, :]
    d = x - centre
    return d * d


def add_sphere(C: np.ndarray, grid: Grid, centre, radius: float) -> None:
    """Add the sub-sampled volume fraction of one sphere to C (in place).

    phi = |x - centre|^2 - radius^2.  Along periodic axes the sphere's cells are
    wrapped into the box (the sphere is evaluated at its unwrapped position and
    the result is stored at the wrapped index), so a drop crossing a periodic
    face is continued on the other side.
    """
    h = grid.h
    n = (grid.nx, grid.ny, grid.nz)
    r2 = radius * radius
    ranges = []
    sq = []
    for a in range(3):
        lo = int(math.floor((centre[a] - radius) / h)) - 1
        hi = int(math.floor((centre[a] + radius) / h)) + 2
        if grid.bc[a] == WALL:
            lo, hi = max(lo, 0), min(hi, n[a])
        ranges.append((lo, hi))
        sq.append(_axis_sq(lo, hi, h, centre[a]))
    dx2, dy2, dz2 = sq
    # (z, sz, y, sy, x, sx) sums in a fixed order: (dx2 + dy2) + dz2
    s = (dx2[None, None, None, None, :, :] + dy2[None, None, :, :, None, None]) \
        + dz2[:, :, None, None, None, None]
    inside = (s < r2).sum(axis=(1, 3, 5)).astype(np.float64) / float(N_SUB ** 3)
    (x0, x1), (y0, y1), (z0, z1) = ranges
    iz = np.arange(z0, z1) % n[2]
    iy = np.arange(y0, y1) % n[1]
    ix = np.arange(x0, x1) % n[0]
    np.add.at(C, (iz[:, None, None], iy[None, :, None], ix[None, None, :]), inside)


def add_cylinder_x(C: np.ndarray, grid: Grid, yc: float, zc: float, radius_of_x) -> None:
    """Sub-sampled volume fraction of a jet along x: phi = (y-yc)^2 + (z-zc)^2 - R(x)^2."""
    h = grid.h
    xs = (np.arange(grid.nx, dtype=np.float64)[:, None] * h + _sub_offsets(h)[None, :])
    R = radius_of_x(xs)  # (nx, N_SUB)
    R2 = R * R
    rmax = float(R.max())
    y0 = max(int(math.floor((yc - rmax) / h)) - 1, 0)
    y1 = min(int(math.floor((yc + rmax) / h)) + 2, grid.ny)
    z0 = max(int(math.floor((zc - rmax) / h)) - 1, 0)
    z1 = min(int(math.floor((zc + rmax) / h)) + 2, grid.nz)
    dy2 = _axis_sq(y0, y1, h, yc)
    dz2 = _axis_sq(z0, z1, h, zc)
    s = dy2[None, None, :, :] + dz2[:, :, None, None]  # (z, sz, y, sy)
    # count over (sz, sy) for each x sub-sample, then sum the x sub-samples
    inside = (s[..., None, None] < R2[None, None, None, None, :, :]).sum(axis=(1, 3, 5))
    C[z0:z1, y0:y1, :] += inside.astype(np.float64) / float(N_SUB ** 3)


def place_spheres(rng, grid: Grid, count: int, rmin: float, rmax: float,
                  gap: float, max_tries: int = 100000):
    """Rejection-sample non-overlapping spheres.

    Radii ~ U[rmin, rmax]; centres uniform in the box, kept at least radius+gap
    from wall faces; two spheres are accepted when their minimum-image distance
    (periodic axes) is at least r_a + r_b + gap.  Returns a list of
    (centre, radius); fewer than ``count`` spheres if the tries run out.
    """
    L = grid.lengths
    out = []
    tries = 0
    while len(out) < count and tries < max_tries:
        tries += 1
        r = rng.uniform(rmin, rmax)
        c = []
        for a in range(3):
            if grid.bc[a] == WALL:
                c.append(rng.uniform(r + gap, L[a] - r - gap))
            else:
                c.append(rng.uniform(0.0, L[a]))
        ok = True
        for (c2, r2) in out:
            d2 = 0.0
            for a in range(3):
                d = c[a] - c2[a]
                if grid.bc[a] == PERIODIC:
                    d -= L[a] * round(d / L[a])
                d2 += d * d
            if d2 < (r + r2 + gap) ** 2:
                ok = False
                break
        if ok:
            out.append((tuple(c), r))
    return out


# ---------------------------------------------------------------- velocity ---

def face_positions(grid: Grid, axis: int):
    """1-D coordinates (x, y, z) of the face centres of the face array normal to ``axis``."""
    h = grid.h
    n = (grid.nx, grid.ny, grid.nz)
    out = []
    for a in range(3):
        if a == axis:
            m = n[a] + (1 if grid.bc[a] == WALL else 0)
            out.append(np.arange(m, dtype=np.float64) * h)          # faces at i*h
        else:
            out.append((np.arange(n[a], dtype=np.float64) + 0.5) * h)  # cell centres
    return out


def zero_wall_faces(grid: Grid, u, v, w) -> None:
    """Set the normal velocity on wall faces to zero (in place)."""
    if grid.bc[0] == WALL:
        u[:, :, 0] = 0.0
        u[:, :, -1] = 0.0
    if grid.bc[1] == WALL:
        v[:, 0, :] = 0.0
        v[:, -1, :] = 0.0
    if grid.bc[2] == WALL:
        w[0, :, :] = 0.0
        w[-1, :, :] = 0.0


def fourier_velocity(rng, grid: Grid, modes: int, kmax: int):
    """u* = sum_m e_m cos(k_m . x + phi_m) at the face centres.

    k_m = 2*pi*(a, b, c)/L with integers |a|, |b|, |c| <= kmax (not all zero),
    e_m a random unit vector, phi_m ~ U[0, 2*pi).
    """
    L = grid.lengths
    ks, es, phis = [], [], []
    for _ in range(modes):
        while True:
            abc = rng.integers(-kmax, kmax + 1, size=3)
            if np.any(abc != 0):
                break
        e = rng.normal(size=3)
        e /= np.linalg.norm(e)
        ks.append([2.0 * math.pi * abc[a] / L[a] for a in range(3)])
        es.append(e)
        phis.append(rng.uniform(0.0, 2.0 * math.pi))
    comps = []
    for axis in range(3):
        x, y, z = face_positions(grid, axis)
        f = np.zeros((z.size, y.size, x.size))
        for k, e, ph in zip(ks, es, phis):
            ex = np.exp(1j * k[0] * x)
            ey = np.exp(1j * k[1] * y)
            ez = np.exp(1j * (k[2] * z + ph))
            P = ez[:, None] * ey[None, :]
            f += e[axis] * (P.real[:, :, None] * ex.real[None, None, :]
                            - P.imag[:, :, None] * ex.imag[None, None, :])
        comps.append(f)
    return comps


def edge_potential_curl(rng, grid: Grid, modes: int, kmax: int):
    """A discretely divergence-free face field: the staggered curl of a random
    Fourier vector potential held on cell edges (periodic axes only).

    A_x lives on x-edges ((i+1/2)h, jh, kh), A_y on ((ih, (j+1/2)h, kh),
    A_z on (ih, jh, (k+1/2)h).  The face velocities are the edge differences
        u = (A_z[j+1] - A_z[j] - A_y[k+1] + A_y[k]) / h
    and cyclically, whose discrete divergence vanishes identically.
    """
    assert all(b == PERIODIC for b in grid.bc)
    h = grid.h
    L = grid.lengths
    nx, ny, nz = grid.nx, grid.ny, grid.nz
    cc = [(np.arange(n) + 0.5) * h for n in (nx, ny, nz)]
    nn = [np.arange(n) * h for n in (nx, ny, nz)]
    A = [np.zeros(grid.shape) for _ in range(3)]
    for _ in range(modes):
        abc = rng.integers(-kmax, kmax + 1, size=3)
        if not np.any(abc != 0):
            abc[0] = 1
        k = [2.0 * math.pi * abc[a] / L[a] for a in range(3)]
        amp = rng.normal(size=3)
        ph = rng.uniform(0.0, 2.0 * math.pi)
        for comp in range(3):
            pos = [nn[0], nn[1], nn[2]]
            pos[comp] = cc[comp]
            x, y, z = pos
            arg = (k[2] * z)[:, None, None] + (k[1] * y)[None, :, None] + (k[0] * x)[None, None, :]
            A[comp] += amp[comp] * np.cos(arg + ph)
    Ax, Ay, Az = A
    rollp = lambda a, ax: np.roll(a, -1, axis=ax)  # value at index+1 (periodic)
    # numpy axes: 0 = z, 1 = y, 2 = x
    u = ((rollp(Az, 1) - Az) - (rollp(Ay, 0) - Ay)) / h
    v = ((rollp(Ax, 0) - Ax) - (rollp(Az, 2) - Az)) / h
    w = ((rollp(Ay, 2) - Ay) - (rollp(Ax, 1) - Ax)) / h
    return u, v, w


# ----------------------------------------------------------- configurations ---

def config1() -> Problem:
    """32^3 triply periodic unit box, one drop R = 0.25 at the centre,
    rho1 = 10 inside, rho2 = 1 outside, u* ~ U[-1, 1] from seed 0, dt = 1e-3."""
    n = 32
    g = Grid(n, n, n, 1.0 / n)
    C = np.zeros(g.shape)
    add_sphere(C, g, (0.5, 0.5, 0.5), 0.25)
    rng = np.random.default_rng(0)
    u = rng.uniform(-1.0, 1.0, size=g.face_shape(0))
    v = rng.uniform(-1.0, 1.0, size=g.face_shape(1))
    w = rng.uniform(-1.0, 1.0, size=g.face_shape(2))
    return Problem("drop32", g, C, u, v, w, rho1=10.0, rho2=1.0, dt=1e-3)


def config2(n: int = 256, drops: int = 64, cfg_id: int = 2, rho1: float = 1000.0) -> Problem:
    """n^3 unit box, periodic in x and y, walls in z, h = 1/n, dt = 1e-4.

    ``drops`` non-overlapping drops, radii ~ U[0.02, 0.08], kept 2h apart and
    2h from the walls; rho1 = 1000 in the drops, rho2 = 1.  u* is 16 random
    Fourier modes (|a|,|b|,|c| <= 4) of unit amplitude plus U[-0.01, 0.01]
    noise, with zero normal velocity on the wall faces.
    """
    g = Grid(n, n, n, 1.0 / n, (PERIODIC, PERIODIC, WALL))
    geo = _rng(cfg_id, 0)
    spheres = place_spheres(geo, g, drops, 0.02, 0.08, 2.0 * g.h)
    C = np.zeros(g.shape)
    for c, r in spheres:
        add_sphere(C, g, c, r)
    u, v, w = fourier_velocity(_rng(cfg_id, 1), g, 16, 4)
    noise = _rng(cfg_id, 2)
    u += noise.uniform(-0.01, 0.01, size=u.shape)
    v += noise.uniform(-0.01, 0.01, size=v.shape)
    w += noise.uniform(-0.01, 0.01, size=w.shape)
    zero_wall_faces(g, u, v, w)
    return Problem(f"drops{n}_walls_z", g, C, u, v, w, rho1=rho1, rho2=1.0, dt=1e-4,
                   extra={"spheres": spheres})


def config3(nx: int = 512, ny: int = 256, nz: int = 256, cfg_id: int = 3) -> Problem:
    """Jet along x in a (2, 1, 1) box, periodic in x, walls in y and z.

    R(x) = 0.08 (1 + 0.05 sum_{i=1..4} sin(m_i pi x + phi_i)), m_i in {2..16};
    u_x = face average of C, plus U[-0.1, 0.1] noise on every component;
    zero normal velocity on the walls; rho1/rho2 = 1000, dt = 5e-5.
    """
    h = 2.0 / nx
    g = Grid(nx, ny, nz, h, (PERIODIC, WALL, WALL))
    geo = _rng(cfg_id, 0)
    m = geo.integers(2, 17, size=4)
    ph = geo.uniform(0.0, 2.0 * math.pi, size=4)

    def radius(x):
        s = np.zeros_like(x)
        for mi, pi_ in zip(m, ph):
            s += np.sin(mi * math.pi * x + pi_)
        return 0.08 * (1.0 + 0.05 * s)

    C = np.zeros(g.shape)
    Ly, Lz = ny * h, nz * h
    add_cylinder_x(C, g, 0.5 * Ly, 0.5 * Lz, radius)
    u = 0.5 * (C + np.roll(C, 1, axis=2))  # x-face i-1/2 between cells i-1 and i
    v = np.zeros(g.face_shape(1))
    w = np.zeros(g.face_shape(2))
    noise = _rng(cfg_id, 2)
    u += noise.uniform(-0.1, 0.1, size=u.shape)
    v += noise.uniform(-0.1, 0.1, size=v.shape)
    w += noise.uniform(-0.1, 0.1, size=w.shape)
    zero_wall_faces(g, u, v, w)
    return Problem(f"jet{nx}x{ny}x{nz}", g, C, u, v, w, rho1=1000.0, rho2=1.0, dt=5e-5,
                   extra={"m": m, "phi": ph})


BATCH_AXES = (32, 48, 64, 96, 128)


def config4(count: int = 256, cfg_id: int = 4, axes=BATCH_AXES):
    """Independent periodic problems of uneven sizes, h = 1/64.

    Each axis size is drawn from ``axes``; 1-8 drops with radii ~ U[0.05, 0.2]
    times the shortest box side (rejection sampling, up to 1000 tries); density
    ratio log-uniform in [1, 1000] with rho2 = 1; u* ~ U[-1, 1]; dt = 1e-3.
    """
    geo = _rng(cfg_id, 0)
    vel = _rng(cfg_id, 1)
    out = []
    for b in range(count):
        nx, ny, nz = (int(geo.choice(axes)) for _ in range(3))
        g = Grid(nx, ny, nz, 1.0 / 64)
        k = int(geo.integers(1, 9))
        Lmin = min(g.lengths)
        spheres = place_spheres(geo, g, k, 0.05 * Lmin, 0.2 * Lmin, 2.0 * g.h, max_tries=1000)
        C = np.zeros(g.shape)
        for c, r in spheres:
            add_sphere(C, g, c, r)
        ratio = float(np.exp(geo.uniform(0.0, math.log(1000.0))))
        u = vel.uniform(-1.0, 1.0, size=g.face_shape(0))
        v = vel.uniform(-1.0, 1.0, size=g.face_shape(1))
        w = vel.uniform(-1.0, 1.0, size=g.face_shape(2))
        out.append(Problem(f"batch{b}_{nx}x{ny}x{nz}", g, C, u, v, w, rho1=ratio, rho2=1.0,
                           dt=1e-3, extra={"spheres": spheres, "requested_drops": k}))
    return out


def config5(n: int = 128, cfg_id: int = 5) -> Problem:
    """n^3 periodic box, one drop of radius 0.2 with a smooth tanh profile
    C = (1 - tanh((r - 0.2)/w))/2, w = 1.5h, rho1/rho2 = 100, u* ~ U[-1, 1];
    the loss target is a discretely divergence-free random Fourier field."""
    g = Grid(n, n, n, 1.0 / n)
    c = (np.arange(n) + 0.5) * g.h - 0.5
    r = np.sqrt(c[:, None, None] ** 2 + c[None, :, None] ** 2 + c[None, None, :] ** 2)
    C = 0.5 * (1.0 - np.tanh((r - 0.2) / (1.5 * g.h)))
    vel = _rng(cfg_id, 1)
    u = vel.uniform(-1.0, 1.0, size=g.face_shape(0))
    v = vel.uniform(-1.0, 1.0, size=g.face_shape(1))
    w = vel.uniform(-1.0, 1.0, size=g.face_shape(2))
    tu, tv, tw = edge_potential_curl(_rng(cfg_id, 3), g, 8, 4)
    scale = 1.0 / max(np.abs(tu).max(), np.abs(tv).max(), np.abs(tw).max())
    return Problem(f"adjoint_drop{n}", g, C, u, v, w, rho1=100.0, rho2=1.0, dt=1e-3,
                   extra={"target": (tu * scale, tv * scale, tw * scale)})


def random_problem(grid: Grid, seed: int, rho1: float = 1000.0, rho2: float = 1.0,
                   dt: float = 1e-3, drops: int = 3) -> Problem:
    """Small seeded problem on any grid (drops of radius ~0.15-0.3 of the box,
    u* ~ U[-1, 1], wall-normal velocity zero) for parity and edge-case tests."""
    rng = np.random.default_rng([100, seed])
    Lmin = min(grid.lengths)
    spheres = place_spheres(rng, grid, drops, 0.15 * Lmin, 0.3 * Lmin, 0.0, max_tries=2000)
    C = np.zeros(grid.shape)
    for c, r in spheres:
        add_sphere(C, grid, c, r)
    np.clip(C, 0.0, 1.0, out=C)
    u = rng.uniform(-1.0, 1.0, size=grid.face_shape(0))
    v = rng.uniform(-1.0, 1.0, size=grid.face_shape(1))
    w = rng.uniform(-1.0, 1.0, size=grid.face_shape(2))
    zero_wall_faces(grid, u, v, w)
    return Problem(f"rand{grid.nx}x{grid.ny}x{grid.nz}_s{seed}", grid, C, u, v, w,
                   rho1=rho1, rho2=rho2, dt=dt, extra={"spheres": spheres})


def random_field(shape, seed: int, mean_free: bool = True) -> np.ndarray:
    """Seeded U[-1, 1] field (optionally with its mean removed) for test potentials."""
    f = np.random.default_rng([200, seed]).uniform(-1.0, 1.0, size=shape)
    if mean_free:
        f -= f.mean()
    return f


def layered_problem(grid: Grid, z_frac: float = 0.41, rho1: float = 1000.0, rho2: float = 1.2,
                    dt: float = 1e-3, g_z: float = -9.81, noise: float = 0.0, seed: int = 0) -> Problem:
    """Fluid 1 below the flat plane z = z_frac * L_z, fluid 2 above (walls in z
    expected), C the exact fraction of each cell below the plane.  u* = dt g_z
    on every z-face off the walls (the predictor's uniform gravity from rest),
    plus U[-noise, noise] on every component; wall-normal velocity zero."""
    h = grid.h
    zi = z_frac * grid.nz * h
    zlo = np.arange(grid.nz) * h
    frac = np.clip((zi - zlo) / h, 0.0, 1.0)
    C = np.broadcast_to(frac[:, None, None], grid.shape).copy()
    u = np.zeros(grid.face_shape(0))
    v = np.zeros(grid.face_shape(1))
    w = np.full(grid.face_shape(2), dt * g_z)
    if noise > 0.0:
        rng = np.random.default_rng([500, seed])
        u += rng.uniform(-noise, noise, size=u.shape)
        v += rng.uniform(-noise, noise, size=v.shape)
        w += rng.uniform(-noise, noise, size=w.shape)
    zero_wall_faces(grid, u, v, w)
    return Problem(f"layered{grid.nx}x{grid.ny}x{grid.nz}", grid, C, u, v, w, rho1=rho1, rho2=rho2, dt=dt,
                   extra={"z_interface": zi, "g_z": g_z})


def drop_curvature(grid: Grid, spheres) -> np.ndarray:
    """Cell curvature field of a set of spheres of fluid 1: kappa = -2/r of
    the sphere whose surface is nearest to the cell centre (minimum image on
    periodic axes), the sign that makes a sphere of fluid 1 of radius r carry
    the Laplace jump 2 sigma / r.  Only its values next to interfaces enter
    the capillary force; elsewhere grad C = 0."""
    L = grid.lengths
    c = [(np.arange(n) + 0.5) * grid.h for n in (grid.nx, grid.ny, grid.nz)]
    best = np.full(grid.shape, np.inf)
    kappa = np.zeros(grid.shape)
    for centre, r in spheres:
        d2 = np.zeros(grid.shape)
        for a, ax in ((0, (None, None, slice(None))), (1, (None, slice(None), None)), (2, (slice(None), None, None))):
            d = c[a] - centre[a]
            if grid.bc[a] == PERIODIC:
                d = d - L[a] * np.round(d / L[a])
            d2 = d2 + (d * d)[ax]
        dist = np.abs(np.sqrt(d2) - r)
        closer = dist < best
        best[closer] = dist[closer]
        kappa[closer] = -2.0 / r
    return kappa
