"""Front-tracking marker function: plain FP64 CPU oracle (numpy on top of the
C oracle).

TEST INFRASTRUCTURE ONLY: only the tests may import this module; the
library's product path never calls it.  Written from Sec. 3.4.2 of the PARIS
paper (arXiv 2012.11744), "Constructing the marker function": the gradient
of the marker function I, spread from the front onto the fixed grid as a
face field G_f (Eq. gradI), is integrated by solving the Poisson equation

    grad^h . grad^h I = grad^h . G_f                    (Eq. FrontMarker3)

on the whole grid (the paper's choice), i.e. the projection's operator with
beta = 1 on every face (0 on wall faces, Sec. 3.8) and the right-hand side
the divergence of G_f (walls carry no flux).  I is fixed up to a constant;
the caller gives its mean (for a front: the volume it encloses over the
domain's), which is the reading taken here since the paper does not say how
the constant is chosen.
"""
from __future__ import annotations

import numpy as np

from . import Operator, cg, divergence, face_shape, remove_mean

WALL = 1


def unit_beta(grid):
    """beta = 1 on every face, 0 on the wall faces."""
    out = []
    for axis in range(3):
        b = np.ones(face_shape(grid, axis))
        if grid.bc[axis] == WALL:
            sl = [slice(None)] * 3
            for end in (0, -1):
                sl[2 - axis] = end
                b[tuple(sl)] = 0.0
        out.append(b)
    return tuple(out)


def marker_function(grid, gx, gy, gz, mean_I, tol=1e-13, max_iter=200000):
    """I with mean(I) = mean_I solving Lap_h I = D G (Eq. FrontMarker3).
    Returns (I, CGResult)."""
    b = divergence(grid, gx, gy, gz, dt=1.0)
    b0 = remove_mean(b)
    op = Operator(grid, *unit_beta(grid))
    res = cg(op, -b0, tol=tol, max_iter=max_iter)  # A = -L: L I = b  <=>  A I = -b
    op.close()
    return remove_mean(res.x) + mean_I, res
