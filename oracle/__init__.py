"""Plain FP64 CPU oracle for the one-fluid pressure projection (ctypes wrapper).

TEST INFRASTRUCTURE ONLY: only the tests, the smoke check and the benchmark's
CPU-baseline arm may import this package.  The library's product path never
calls it.  The arithmetic lives in ``paris_oracle.c`` (plain C, IEEE double,
no fused multiply-add); this module marshals numpy arrays and adds the two
steps that are plain library calls (Lanczos eigenvalues of the CG tridiagonal).

Every function follows a passage of the PARIS paper (arXiv 2012.11744):
  face_coeffs      Eq. muH and the 1/rho coefficients of Sec. 3.7.1; walls Sec. 3.8
  divergence       Eqs. cont2 / incompdisc3, divided by dt
  assemble         the A1..A7 system form of Sec. 3.7.1 (as the CSR of -L)
  cg               solves Eq. poisson (unpreconditioned conjugate gradients)
  project          Eq. fotm
  projection_step  steps 1-6 in order, then mean(p) = 0
  project_adjoint / face_coeffs_adjoint: derivatives of the above (no paper
  counterpart; pinned against central finite differences in the tests)

Solid cells (the "Lego" solids of Sec. 3.8: link flags that block the
velocity and zero the pressure coefficients on the solid and its boundary)
are in ``solid.py``.  The implicit viscous step of Sec. 3.2.3 (Eq. muelliptic) is in ``viscous.py``
(numpy and scipy.sparse, FP64); the capillary (Eq. csf2) and gravity forcing
of the predictor (Eq. nonconspredictedvel) in ``forcing.py`` (numpy, FP64);
the free-surface projections of Sec. 3.7.5 (the ghost-fluid Dirichlet solve
in the liquid and the phantom projection in two gas layers) in
``freesurf.py`` (numpy and scipy.sparse, FP64).
"""
from __future__ import annotations

import ctypes as ct
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "paris_oracle.c")
_LIB = os.path.join(_HERE, "libparis_oracle.so")
_lock = threading.Lock()
_lib = None

PERIODIC = 0
WALL = 1


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP, -ffp-contract=off)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-std=c99",
                               "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Grid(ct.Structure):
    _fields_ = [("nx", ct.c_int), ("ny", ct.c_int), ("nz", ct.c_int), ("h", ct.c_double),
                ("bc", ct.c_int * 3)]


class _CGStats(ct.Structure):
    _fields_ = [("iters", ct.c_int), ("stagnated", ct.c_int), ("rel_res_l2", ct.c_double),
                ("rel_res_linf", ct.c_double), ("n_coef", ct.c_int)]


_D = ct.POINTER(ct.c_double)


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ct.CDLL(build())
            G = ct.POINTER(_Grid)
            P = ct.c_void_p
            lib.oracle_face_count.argtypes = [G, ct.c_int]
            lib.oracle_face_count.restype = ct.c_int64
            lib.oracle_face_coeffs.argtypes = [G, _D, ct.c_double, ct.c_double, _D, _D, _D]
            lib.oracle_divergence.argtypes = [G, _D, _D, _D, ct.c_double, _D]
            lib.oracle_assemble.argtypes = [G, _D, _D, _D]
            lib.oracle_assemble.restype = P
            lib.oracle_csr_free.argtypes = [P]
            lib.oracle_csr_nnz.argtypes = [P]
            lib.oracle_csr_nnz.restype = ct.c_int64
            lib.oracle_csr_export.argtypes = [P, ct.POINTER(ct.c_int64), ct.POINTER(ct.c_int32), _D]
            lib.oracle_csr_matvec.argtypes = [P, _D, _D]
            lib.oracle_cg.argtypes = [P, _D, _D, ct.c_double, ct.c_int, ct.c_int, _D, ct.c_int,
                                      ct.POINTER(_CGStats)]
            lib.oracle_project.argtypes = [G, _D, _D, _D, _D, ct.c_double, _D, _D, _D]
            lib.oracle_face_gradient.argtypes = [G, _D, _D, _D, _D]
            lib.oracle_remove_mean.argtypes = [ct.c_int64, _D]
            lib.oracle_null_project.argtypes = [ct.c_int64, _D, ct.c_void_p]
            lib.oracle_cg_masked.argtypes = [P, _D, _D, ct.c_double, ct.c_int, ct.c_int, _D, ct.c_int,
                                             ct.c_void_p, ct.POINTER(_CGStats)]
            lib.oracle_sum.argtypes = [ct.c_int64, _D]
            lib.oracle_sum.restype = ct.c_double
            lib.oracle_dot.argtypes = [ct.c_int64, _D, _D]
            lib.oracle_dot.restype = ct.c_double
            lib.oracle_project_adjoint.argtypes = [G, P, _D, _D, _D, _D, ct.c_double, _D, _D, _D,
                                                   _D, _D, _D, _D, _D, _D, _D, ct.c_double, ct.c_int,
                                                   ct.POINTER(_CGStats)]
            lib.oracle_face_coeffs_adjoint.argtypes = [G, ct.c_double, ct.c_double, _D, _D, _D,
                                                       _D, _D, _D, _D]
            _lib = lib
    return _lib


def _g(grid) -> _Grid:
    g = _Grid()
    g.nx, g.ny, g.nz, g.h = int(grid.nx), int(grid.ny), int(grid.nz), float(grid.h)
    for a in range(3):
        g.bc[a] = int(grid.bc[a])
    return g


def _p(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_D)


def _c(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def face_shape(grid, axis):
    n = [grid.nz, grid.ny, grid.nx]
    n[2 - axis] += 1 if grid.bc[axis] == WALL else 0
    return tuple(n)


# ------------------------------------------------------------------ steps ---

def face_coeffs(grid, C, rho1, rho2):
    """beta_x, beta_y, beta_z (face arrays) from the cell volume fraction C."""
    lib = _load()
    C = _c(C)
    out = [np.empty(face_shape(grid, a)) for a in range(3)]
    g = _g(grid)
    lib.oracle_face_coeffs(ct.byref(g), _p(C), float(rho1), float(rho2), *(_p(o) for o in out))
    return tuple(out)


def divergence(grid, u, v, w, dt=1.0):
    """b = (grad^h . u)/dt at the cell centres (mean not removed)."""
    lib = _load()
    u, v, w = _c(u), _c(v), _c(w)
    out = np.empty((grid.nz, grid.ny, grid.nx))
    g = _g(grid)
    lib.oracle_divergence(ct.byref(g), _p(u), _p(v), _p(w), float(dt), _p(out))
    return out


def remove_mean(x):
    lib = _load()
    x = _c(x).copy()
    lib.oracle_remove_mean(x.size, _p(x))
    return x


def mean(x):
    lib = _load()
    x = _c(x)
    return lib.oracle_sum(x.size, _p(x)) / x.size


def face_gradient(grid, p):
    lib = _load()
    p = _c(p)
    out = [np.empty(face_shape(grid, a)) for a in range(3)]
    g = _g(grid)
    lib.oracle_face_gradient(ct.byref(g), _p(p), *(_p(o) for o in out))
    return tuple(out)


class Operator:
    """The assembled CSR matrix A = -L of the variable-coefficient Poisson operator."""

    def __init__(self, grid, bx, by, bz):
        self.lib = _load()
        self.grid = grid
        self._keep = [_c(bx), _c(by), _c(bz)]
        g = _g(grid)
        self.ptr = self.lib.oracle_assemble(ct.byref(g), *(_p(b) for b in self._keep))
        self.n = grid.nx * grid.ny * grid.nz

    def close(self):
        if self.ptr:
            self.lib.oracle_csr_free(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def csr(self):
        """(rowptr, col, val) numpy copies of the assembled matrix."""
        nnz = self.lib.oracle_csr_nnz(self.ptr)
        rowptr = np.empty(self.n + 1, np.int64)
        col = np.empty(nnz, np.int32)
        val = np.empty(nnz, np.float64)
        self.lib.oracle_csr_export(self.ptr, rowptr.ctypes.data_as(ct.POINTER(ct.c_int64)),
                                   col.ctypes.data_as(ct.POINTER(ct.c_int32)), _p(val))
        return rowptr, col, val

    def apply(self, x):
        """A x = -L x for a cell field x."""
        x = _c(x)
        y = np.empty_like(x)
        self.lib.oracle_csr_matvec(self.ptr, _p(x), _p(y))
        return y

    def apply_L(self, x):
        """L x = grad^h . (beta grad^h x)."""
        return -self.apply(x)


@dataclass
class CGResult:
    x: np.ndarray
    iters: int
    stagnated: bool
    rel_res_l2: float
    rel_res_linf: float
    alphas: np.ndarray
    betas: np.ndarray

    def lanczos_extremes(self):
        """(lambda_min, lambda_max) estimates of A on the Krylov space from the CG
        coefficients: T_kk = 1/alpha_k + beta_{k-1}/alpha_{k-1},
        T_k,k+1 = sqrt(beta_k)/alpha_k (the Lanczos-CG correspondence)."""
        a, b = self.alphas, self.betas
        m = len(a)
        if m == 0:
            return (np.nan, np.nan)
        d = np.empty(m)
        e = np.empty(max(m - 1, 0))
        for k in range(m):
            d[k] = 1.0 / a[k] + (b[k - 1] / a[k - 1] if k > 0 else 0.0)
            if k < m - 1:
                e[k] = np.sqrt(b[k]) / a[k]
        T = np.diag(d) + np.diag(e, 1) + np.diag(e, -1)
        ev = np.linalg.eigvalsh(T)
        return float(ev[0]), float(ev[-1])


def null_project(x, fluid=None):
    """Remove the null-space part of x: the mean (no solid), or with a solid
    mask (fluid = 1 outside the solid, Sec. 3.8) the mean over the fluid
    cells, and 0 in the solid cells."""
    lib = _load()
    x = _c(x).copy()
    fl = None if fluid is None else np.ascontiguousarray(fluid, dtype=np.uint8)
    lib.oracle_null_project(x.size, _p(x), None if fl is None else fl.ctypes.data)
    return x


def cg(op: Operator, rhs, x0=None, tol=1e-13, max_iter=200000, check=50, keep_coef=4000, fluid=None):
    """Unpreconditioned CG on A x = rhs (rhs must be orthogonal to the null
    space: mean-free, and with a solid mask zero in the solid cells)."""
    lib = op.lib
    rhs = _c(rhs)
    x = np.zeros_like(rhs) if x0 is None else _c(x0).copy()
    coef = np.zeros(2 * keep_coef)
    st = _CGStats()
    fl = None if fluid is None else np.ascontiguousarray(fluid, dtype=np.uint8)
    lib.oracle_cg_masked(op.ptr, _p(rhs), _p(x), float(tol), int(max_iter), int(check), _p(coef),
                         int(keep_coef), None if fl is None else fl.ctypes.data, ct.byref(st))
    nc = st.n_coef
    return CGResult(x, st.iters, bool(st.stagnated), st.rel_res_l2, st.rel_res_linf,
                    coef[0:2 * nc:2].copy(), coef[1:2 * nc:2].copy())


def project(grid, bx, by, bz, p, dt, u, v, w):
    """u = u* - dt beta (grad^h p) on every non-wall face; wall faces set to 0."""
    lib = _load()
    out = [_c(u).copy(), _c(v).copy(), _c(w).copy()]
    g = _g(grid)
    lib.oracle_project(ct.byref(g), _p(_c(bx)), _p(_c(by)), _p(_c(bz)), _p(_c(p)), float(dt),
                       *(_p(o) for o in out))
    return tuple(out)


@dataclass
class Projection:
    beta: tuple
    rhs: np.ndarray          # b = D u*/dt before mean removal
    mean_b: float            # removed mean of b
    p: np.ndarray            # mean-free pressure
    u: tuple                 # corrected velocity
    cg: CGResult
    op: Operator


def projection_step(grid, C, rho1, rho2, dt, u, v, w, tol=1e-13, max_iter=200000, p0=None):
    """One full projection: beta from C, b = D u*/dt, mean removal, solve
    L p = b with mean(p) = 0, correct u.  Returns a Projection record."""
    beta = face_coeffs(grid, C, rho1, rho2)
    b = divergence(grid, u, v, w, dt)
    mb = mean(b)
    b0 = remove_mean(b)
    op = Operator(grid, *beta)
    # A = -L, so L p = b  <=>  A p = -b
    res = cg(op, -b0, x0=p0, tol=tol, max_iter=max_iter)
    p = remove_mean(res.x)
    uu = project(grid, *beta, p, dt, u, v, w)
    return Projection(beta, b, mb, p, uu, res, op)


def project_adjoint(grid, op: Operator, beta, p, dt, gu, gv, gw, tol=1e-13, max_iter=200000):
    """Adjoint of the projection: returns (dL/du*, dL/dbeta, q, CGResult-like stats)."""
    lib = op.lib
    gin = [_c(gu), _c(gv), _c(gw)]
    gstar = [np.empty_like(a) for a in gin]
    gbeta = [np.empty_like(a) for a in gin]
    q = np.empty((grid.nz, grid.ny, grid.nx))
    st = _CGStats()
    g = _g(grid)
    bx, by, bz = (_c(b) for b in beta)
    lib.oracle_project_adjoint(ct.byref(g), op.ptr, _p(bx), _p(by), _p(bz), _p(_c(p)), float(dt),
                               *(_p(a) for a in gin), *(_p(a) for a in gstar),
                               *(_p(a) for a in gbeta), _p(q), float(tol), int(max_iter),
                               ct.byref(st))
    return tuple(gstar), tuple(gbeta), q, st


def face_coeffs_adjoint(grid, rho1, rho2, beta, gbeta):
    """dL/dC from dL/dbeta through beta = 1/rho_f."""
    lib = _load()
    gC = np.empty((grid.nz, grid.ny, grid.nx))
    g = _g(grid)
    bx, by, bz = (_c(b) for b in beta)
    gx, gy, gz = (_c(b) for b in gbeta)
    lib.oracle_face_coeffs_adjoint(ct.byref(g), float(rho1), float(rho2), _p(bx), _p(by), _p(bz),
                                   _p(gx), _p(gy), _p(gz), _p(gC))
    return gC
