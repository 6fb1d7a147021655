"""Python binding of the projection library: torch tensors in, C ABI calls out.

Only argument marshalling happens here (shape/dtype/device checks, data
pointers, the current CUDA stream); every step of the projection runs in the
CUDA kernels of libparis.so.  The call names follow include/paris.h.
"""
from __future__ import annotations

import ctypes as ct
from dataclasses import dataclass

import numpy as np
import torch

from . import _abi
from ._abi import (MIXED, FP64, PERIODIC, WALL, SMOOTH_JACOBI, SMOOTH_RBGS,  # noqa: F401
                   SMOOTH_RBGS_2PASS, ParisError)


@dataclass
class Grid:
    """nx*ny*nz cubic cells of edge h; bc per axis: PERIODIC (0) or WALL (1)."""
    nx: int
    ny: int
    nz: int
    h: float
    bc: tuple = (PERIODIC, PERIODIC, PERIODIC)

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)

    def face_shape(self, axis: int):
        n = [self.nz, self.ny, self.nx]
        n[2 - axis] += 1 if self.bc[axis] == WALL else 0
        return tuple(n)


def default_opts(**kw) -> _abi.Opts:
    lib = _abi.load()
    o = _abi.Opts()
    lib.paris_default_opts(ct.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise AttributeError(f"unknown option {k}")
        setattr(o, k, v)
    return o


def launch_count() -> int:
    """Number of CUDA kernels libparis.so has launched in this process."""
    return int(_abi.load().paris_launch_count())


def check_arithmetic(v, shift: int = 0) -> int:
    """paris_check_arithmetic on a contiguous FP64 CUDA tensor: the number of
    values where the library's integer FP64<->FP32 conversions (scaled by
    2^shift) or its FP64 reciprocal disagree with the GPU's instructions."""
    if not (isinstance(v, torch.Tensor) and v.is_cuda and v.dtype == torch.float64 and v.is_contiguous()):
        raise TypeError("v must be a contiguous float64 CUDA tensor")
    out = ct.c_int64(-1)
    stream = torch.cuda.current_stream(v.device).cuda_stream
    _abi.check(_abi.load().paris_check_arithmetic(ct.c_void_p(v.data_ptr()), v.numel(), int(shift),
                                                  ct.byref(out), ct.c_void_p(stream)),
               "paris_check_arithmetic")
    return int(out.value)


def stream_rates(a, b, c, o, reps: int = 5) -> tuple:
    """paris_stream_rates on four contiguous float32 CUDA tensors of one size
    (a, b, c read; o overwritten): (read-only GB/s, triad GB/s)."""
    ts = (a, b, c, o)
    if not all(isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()
               and t.numel() == a.numel() for t in ts):
        raise TypeError("a, b, c, o must be contiguous float32 CUDA tensors of one size")
    rd, tr = ct.c_double(0.0), ct.c_double(0.0)
    stream = torch.cuda.current_stream(a.device).cuda_stream
    _abi.check(_abi.load().paris_stream_rates(*(ct.c_void_p(t.data_ptr()) for t in ts), a.numel(), int(reps),
                                              ct.byref(rd), ct.byref(tr), ct.c_void_p(stream)),
               "paris_stream_rates")
    return rd.value, tr.value


def _grid_struct(g) -> _abi.Grid:
    s = _abi.Grid()
    s.nx, s.ny, s.nz, s.h = int(g.nx), int(g.ny), int(g.nz), float(g.h)
    for a in range(3):
        s.bc[a] = int(g.bc[a])
    return s


class Context:
    """One paris_ctx: a grid, solver options, device workspace and a stream.

    ``stream``: a torch.cuda.Stream (default: the current stream at creation).
    All tensors passed to the methods must be float64, contiguous and on the
    context's device.
    """

    def __init__(self, grid, opts: _abi.Opts | None = None, device=None, stream=None, **kw):
        self.lib = _abi.load()
        self.grid = Grid(grid.nx, grid.ny, grid.nz, grid.h, tuple(grid.bc))
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else
                                   torch.device(device).index or 0)
        with torch.cuda.device(self.device):
            self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.opts = opts if opts is not None else default_opts(**kw)
        self._ptr = ct.c_void_p()
        gs = _grid_struct(self.grid)
        with torch.cuda.device(self.device):
            _abi.check(self.lib.paris_create(ct.byref(self._ptr), ct.byref(gs), ct.byref(self.opts),
                                             ct.c_void_p(self.stream.cuda_stream)), "paris_create")

    # ------------------------------------------------------------ lifetime
    def close(self):
        if getattr(self, "_ptr", None) and self._ptr.value:
            self.lib.paris_destroy(self._ptr)
            self._ptr = ct.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def set_opts(self, opts=None, **kw):
        o = opts if opts is not None else self.opts
        for k, v in kw.items():
            setattr(o, k, v)
        _abi.check(self.lib.paris_set_opts(self._ptr, ct.byref(o)), "paris_set_opts")
        self.opts = o

    # ------------------------------------------------------------- helpers
    def _t(self, x: torch.Tensor, shape, name: str) -> ct.c_void_p:
        if not isinstance(x, torch.Tensor):
            raise TypeError(f"{name}: expected a torch.Tensor")
        if x.dtype != torch.float64 or not x.is_contiguous() or x.device != self.device:
            raise ValueError(f"{name}: need a contiguous float64 tensor on {self.device}")
        if tuple(x.shape) != tuple(shape) and x.numel() != int(np.prod(shape)):
            raise ValueError(f"{name}: shape {tuple(x.shape)} != {tuple(shape)}")
        return ct.c_void_p(x.data_ptr())

    def empty_cells(self):
        return torch.empty(self.grid.shape, dtype=torch.float64, device=self.device)

    def empty_faces(self):
        return tuple(torch.empty(self.grid.face_shape(a), dtype=torch.float64, device=self.device)
                     for a in range(3))

    # --------------------------------------------------------------- steps
    def face_coeffs(self, C, rho1, rho2, out=None):
        """beta_f = 1/rho_f (Eq. muH, arithmetic face density), 0 on walls."""
        bx, by, bz = out if out is not None else self.empty_faces()
        g = self.grid
        _abi.check(self.lib.paris_face_coeffs(self._ptr, self._t(C, g.shape, "C"), float(rho1),
                                              float(rho2), self._t(bx, g.face_shape(0), "beta_x"),
                                              self._t(by, g.face_shape(1), "beta_y"),
                                              self._t(bz, g.face_shape(2), "beta_z")),
                   "paris_face_coeffs")
        return bx, by, bz

    def divergence(self, u, v, w, dt, out=None, want_mean=True):
        """rhs = (grad^h . u)/dt with its mean removed; returns (rhs, mean)."""
        g = self.grid
        rhs = out if out is not None else self.empty_cells()
        mean = ct.c_double(0.0)
        _abi.check(self.lib.paris_divergence(self._ptr, self._t(u, g.face_shape(0), "u"),
                                             self._t(v, g.face_shape(1), "v"),
                                             self._t(w, g.face_shape(2), "w"), float(dt),
                                             self._t(rhs, g.shape, "rhs"),
                                             ct.byref(mean) if want_mean else None),
                   "paris_divergence")
        return rhs, mean.value

    def poisson_solve(self, bx, by, bz, rhs, p, check=True):
        """Solve grad^h.(beta grad^h p) = rhs (mean(p) = 0); p in/out. Returns stats dict."""
        g = self.grid
        st = _abi.Stats()
        s = self.lib.paris_poisson_solve(self._ptr, self._t(bx, g.face_shape(0), "beta_x"),
                                         self._t(by, g.face_shape(1), "beta_y"),
                                         self._t(bz, g.face_shape(2), "beta_z"),
                                         self._t(rhs, g.shape, "rhs"), self._t(p, g.shape, "p"),
                                         ct.byref(st))
        if check:
            _abi.check(s, "paris_poisson_solve", st.as_dict())
        d = st.as_dict()
        d["status"] = s
        return d

    def project(self, bx, by, bz, p, dt, u, v, w):
        """u <- u - dt beta grad^h p on non-wall faces (Eq. fotm), wall faces 0."""
        g = self.grid
        _abi.check(self.lib.paris_project(self._ptr, self._t(bx, g.face_shape(0), "beta_x"),
                                          self._t(by, g.face_shape(1), "beta_y"),
                                          self._t(bz, g.face_shape(2), "beta_z"),
                                          self._t(p, g.shape, "p"), float(dt),
                                          self._t(u, g.face_shape(0), "u"),
                                          self._t(v, g.face_shape(1), "v"),
                                          self._t(w, g.face_shape(2), "w")), "paris_project")

    def projection_step(self, C, rho1, rho2, dt, u, v, w, p, check=True):
        """The four steps on device tensors; u, v, w, p updated in place."""
        g = self.grid
        st = _abi.Stats()
        s = self.lib.paris_projection_step(self._ptr, self._t(C, g.shape, "C"), float(rho1),
                                           float(rho2), float(dt),
                                           self._t(u, g.face_shape(0), "u"),
                                           self._t(v, g.face_shape(1), "v"),
                                           self._t(w, g.face_shape(2), "w"),
                                           self._t(p, g.shape, "p"), ct.byref(st))
        if check:
            _abi.check(s, "paris_projection_step", st.as_dict())
        d = st.as_dict()
        d["status"] = s
        return d

    def set_solid(self, s):
        """Solid cells (Sec. 3.8): s a uint8 tensor of the cell shape on the
        context's device, nonzero = fluid, or None to clear.  The context
        keeps a reference to s while it is set."""
        g = self.grid
        if s is None:
            _abi.check(self.lib.paris_set_solid(self._ptr, ct.c_void_p(None)), "paris_set_solid")
            self._solid = None
            return
        n = int(np.prod(g.shape))
        if s.dtype != torch.uint8 or not s.is_contiguous() or s.device != self.device or s.numel() != n:
            raise ValueError(f"s: need a contiguous uint8 tensor of {n} cells on {self.device}")
        _abi.check(self.lib.paris_set_solid(self._ptr, ct.c_void_p(s.data_ptr())), "paris_set_solid")
        self._solid = s

    def marker_function(self, gx, gy, gz, mean_I, I=None, check=True):
        """Front-tracking marker function (Eq. FrontMarker3): Lap_h I = D G with
        mean(I) = mean_I; I (cells) is the initial guess when given.  Returns
        (I, stats dict)."""
        g = self.grid
        I = I if I is not None else torch.zeros(g.shape, dtype=torch.float64, device=self.device)
        st = _abi.Stats()
        s = self.lib.paris_marker_function(self._ptr, self._t(gx, g.face_shape(0), "gx"),
                                           self._t(gy, g.face_shape(1), "gy"),
                                           self._t(gz, g.face_shape(2), "gz"), float(mean_I),
                                           self._t(I, g.shape, "I"), ct.byref(st))
        if check:
            _abi.check(s, "paris_marker_function", st.as_dict())
        d = st.as_dict()
        d["status"] = s
        return I, d

    def free_surface_step(self, C, rho_l, dt, u, v, w, p, p_gas=None, theta=None, kappa=None, sigma=0.0,
                          check=True):
        """Free-surface projection (Sec. 3.7.5): solved in the liquid (C < 1/2,
        C the gas fraction), the gas a Dirichlet condition p_s = p_gas +
        sigma (kappa_c + kappa_g)/2 at theta h from the liquid node (theta: three
        face tensors or None for 1).  u, v, w, p in place; p_gas, kappa may be
        None (0).  Returns the stats dict."""
        g = self.grid
        st = _abi.Stats()
        none = ct.c_void_p(None)
        th = [none] * 3 if theta is None else [self._t(t, g.face_shape(a), f"theta_{'xyz'[a]}")
                                               for a, t in enumerate(theta)]
        pg = none if p_gas is None else self._t(p_gas, g.shape, "p_gas")
        kp = none if kappa is None else self._t(kappa, g.shape, "kappa")
        s = self.lib.paris_free_surface_step(self._ptr, self._t(C, g.shape, "C"), float(rho_l), float(dt), *th, kp,
                                             float(sigma), pg, self._t(u, g.face_shape(0), "u"),
                                             self._t(v, g.face_shape(1), "v"), self._t(w, g.face_shape(2), "w"),
                                             self._t(p, g.shape, "p"), ct.byref(st))
        if check:
            _abi.check(s, "paris_free_surface_step", st.as_dict())
        d = st.as_dict()
        d["status"] = s
        return d

    def phantom_projection(self, C, u, v, w, phat=None, check=True):
        """Phantom projection in the first two gas layers (Sec. 3.7.5,
        "Ensuring volume conservation"): u, v, w in place; returns (phat,
        stats dict)."""
        g = self.grid
        phat = phat if phat is not None else torch.zeros(g.shape, dtype=torch.float64, device=self.device)
        st = _abi.Stats()
        s = self.lib.paris_phantom_projection(self._ptr, self._t(C, g.shape, "C"), self._t(u, g.face_shape(0), "u"),
                                              self._t(v, g.face_shape(1), "v"), self._t(w, g.face_shape(2), "w"),
                                              self._t(phat, g.shape, "phat"), ct.byref(st))
        if check:
            _abi.check(s, "paris_phantom_projection", st.as_dict())
        d = st.as_dict()
        d["status"] = s
        return phat, d

    def predictor_forcing(self, C, kappa, rho1, rho2, sigma, gravity, tau, u, v, w, beta=None):
        """Capillary (CSF) and gravity forcing of the predictor: u, v, w (in
        u^n, out u* = u^n + tau a_f) in place; returns the face coefficients
        (written to ``beta`` when given).  kappa may be None (0)."""
        g = self.grid
        bx, by, bz = beta if beta is not None else self.empty_faces()
        kp = ct.c_void_p(None) if kappa is None else self._t(kappa, g.shape, "kappa")
        gx, gy, gz = (float(x) for x in gravity)
        _abi.check(self.lib.paris_predictor_forcing(self._ptr, self._t(C, g.shape, "C"), kp, float(rho1),
                                                    float(rho2), float(sigma), gx, gy, gz, float(tau),
                                                    self._t(u, g.face_shape(0), "u"),
                                                    self._t(v, g.face_shape(1), "v"),
                                                    self._t(w, g.face_shape(2), "w"),
                                                    self._t(bx, g.face_shape(0), "beta_x"),
                                                    self._t(by, g.face_shape(1), "beta_y"),
                                                    self._t(bz, g.face_shape(2), "beta_z")),
                   "paris_predictor_forcing")
        return bx, by, bz

    def projection_step_forced(self, C, kappa, rho1, rho2, sigma, gravity, dt, u, v, w, p, check=True):
        """Forcing (tau = dt) fused into the projection step: u, v, w in u^n,
        out u^{n+1}; p in: initial guess, out: the pressure."""
        g = self.grid
        st = _abi.Stats()
        kp = ct.c_void_p(None) if kappa is None else self._t(kappa, g.shape, "kappa")
        gx, gy, gz = (float(x) for x in gravity)
        s = self.lib.paris_projection_step_forced(self._ptr, self._t(C, g.shape, "C"), kp, float(rho1),
                                                  float(rho2), float(sigma), gx, gy, gz, float(dt),
                                                  self._t(u, g.face_shape(0), "u"),
                                                  self._t(v, g.face_shape(1), "v"),
                                                  self._t(w, g.face_shape(2), "w"),
                                                  self._t(p, g.shape, "p"), ct.byref(st))
        if check:
            _abi.check(s, "paris_projection_step_forced", st.as_dict())
        d = st.as_dict()
        d["status"] = s
        return d

    def projection_step_host(self, C, rho1, rho2, dt, u, v, w, p, check=True):
        """The four steps on HOST arrays (numpy float64 or CPU torch tensors,
        ideally pinned); u, v, w, p updated in place."""
        g = self.grid

        def hp(x, shape, name):
            if isinstance(x, torch.Tensor):
                if x.device.type != "cpu" or x.dtype != torch.float64 or not x.is_contiguous():
                    raise ValueError(f"{name}: need a contiguous float64 CPU tensor")
                ptr = x.data_ptr()
                n = x.numel()
            else:
                if x.dtype != np.float64 or not x.flags.c_contiguous:
                    raise ValueError(f"{name}: need a contiguous float64 array")
                ptr = x.ctypes.data
                n = x.size
            if n != int(np.prod(shape)):
                raise ValueError(f"{name}: size {n} != {shape}")
            return ct.c_void_p(ptr)

        st = _abi.Stats()
        s = self.lib.paris_projection_step_host(self._ptr, hp(C, g.shape, "C"), float(rho1),
                                                float(rho2), float(dt), hp(u, g.face_shape(0), "u"),
                                                hp(v, g.face_shape(1), "v"),
                                                hp(w, g.face_shape(2), "w"), hp(p, g.shape, "p"),
                                                ct.byref(st))
        if check:
            _abi.check(s, "paris_projection_step_host", st.as_dict())
        d = st.as_dict()
        d["status"] = s
        return d

    def project_adjoint(self, bx, by, bz, p, dt, gu, gv, gw, q=None, check=True):
        """Adjoint of the projection: returns ((gus, gvs, gws), (gbx, gby, gbz), q, stats)
        with gus = dLoss/du* and gb = dLoss/dbeta for g = dLoss/du."""
        g = self.grid
        gus, gbt = self.empty_faces(), self.empty_faces()
        if q is None:
            q = torch.zeros(g.shape, dtype=torch.float64, device=self.device)
        st = _abi.Stats()
        fs = [g.face_shape(a) for a in range(3)]
        s = self.lib.paris_project_adjoint(
            self._ptr, self._t(bx, fs[0], "beta_x"), self._t(by, fs[1], "beta_y"),
            self._t(bz, fs[2], "beta_z"), self._t(p, g.shape, "p"), float(dt),
            self._t(gu, fs[0], "gu"), self._t(gv, fs[1], "gv"), self._t(gw, fs[2], "gw"),
            *(self._t(x, fs[a], "gus") for a, x in enumerate(gus)),
            *(self._t(x, fs[a], "gbeta") for a, x in enumerate(gbt)),
            self._t(q, g.shape, "q"), ct.byref(st))
        if check:
            _abi.check(s, "paris_project_adjoint", st.as_dict())
        d = st.as_dict()
        d["status"] = s
        return gus, gbt, q, d

    def face_coeffs_adjoint(self, rho1, rho2, bx, by, bz, gbx, gby, gbz, out=None):
        """dLoss/dC from dLoss/dbeta (cells)."""
        g = self.grid
        gC = out if out is not None else self.empty_cells()
        fs = [g.face_shape(a) for a in range(3)]
        _abi.check(self.lib.paris_face_coeffs_adjoint(
            self._ptr, float(rho1), float(rho2), self._t(bx, fs[0], "beta_x"),
            self._t(by, fs[1], "beta_y"), self._t(bz, fs[2], "beta_z"),
            self._t(gbx, fs[0], "gbeta_x"), self._t(gby, fs[1], "gbeta_y"),
            self._t(gbz, fs[2], "gbeta_z"), self._t(gC, g.shape, "gC")), "paris_face_coeffs_adjoint")
        return gC

    def face_viscosity(self, comp, C, mu1, mu2, rho1, rho2, out=None):
        """nu_f = (mu_L + mu_R)/(rho_L + rho_R) on the faces of component comp
        (Eq. muH in both cells), 0 on its wall faces."""
        g = self.grid
        fs = g.face_shape(comp)
        nu = out if out is not None else torch.empty(fs, dtype=torch.float64, device=self.device)
        _abi.check(self.lib.paris_face_viscosity(self._ptr, int(comp), self._t(C, g.shape, "C"), float(mu1),
                                                 float(mu2), float(rho1), float(rho2), self._t(nu, fs, "nu")),
                   "paris_face_viscosity")
        return nu

    def viscous_solve(self, comp, nu, tau, un, us=None, tol=1e-12, max_iter=10000, check=True, multigrid=False):
        """u* - tau nu Lap_h u* = u^n for component comp (Eq. muelliptic) on its
        face array; returns (us, stats dict).  multigrid: the V-cycle-
        preconditioned flexible CG (paris_viscous_solve_mg) instead of the
        Jacobi-preconditioned CG."""
        g = self.grid
        fs = g.face_shape(comp)
        us = us if us is not None else torch.empty(fs, dtype=torch.float64, device=self.device)
        st = _abi.Stats()
        fn = self.lib.paris_viscous_solve_mg if multigrid else self.lib.paris_viscous_solve
        s = fn(self._ptr, int(comp), self._t(nu, fs, "nu"), float(tau), self._t(un, fs, "un"),
               self._t(us, fs, "us"), float(tol), int(max_iter), ct.byref(st))
        if check:
            _abi.check(s, "paris_viscous_solve_mg" if multigrid else "paris_viscous_solve", st.as_dict())
        d = st.as_dict()
        d["status"] = s
        return us, d

    def residual_norms(self, bx, by, bz, rhs, p):
        """FP64 (||rhs - L p||_2/||rhs||_2, ||.||_inf/||rhs||_inf) on the device."""
        g = self.grid
        a, b = ct.c_double(), ct.c_double()
        _abi.check(self.lib.paris_residual_norms(self._ptr, self._t(bx, g.face_shape(0), "beta_x"),
                                                 self._t(by, g.face_shape(1), "beta_y"),
                                                 self._t(bz, g.face_shape(2), "beta_z"),
                                                 self._t(rhs, g.shape, "rhs"),
                                                 self._t(p, g.shape, "p"), ct.byref(a), ct.byref(b)),
                   "paris_residual_norms")
        return a.value, b.value

    def profile(self, enable: bool = True):
        """Start (clearing the counters) or stop per-kernel-class event timing."""
        _abi.check(self.lib.paris_profile(self._ptr, 1 if enable else 0), "paris_profile")

    def profile_read(self):
        """{class name: {launches, timed, ms, bytes}} for the instrumented classes."""
        out = {}
        for k, name in enumerate(_abi.K_NAMES):
            kp = _abi.KernelProf()
            _abi.check(self.lib.paris_profile_read(self._ptr, k, ct.byref(kp)), "paris_profile_read")
            out[name] = {"launches": kp.launches, "timed": kp.timed, "ms": kp.ms, "bytes": kp.bytes}
        return out

    def max_divergence(self, u, v, w):
        """max |grad^h . u| over the cells, computed on the device."""
        g = self.grid
        m = ct.c_double()
        _abi.check(self.lib.paris_max_divergence(self._ptr, self._t(u, g.face_shape(0), "u"),
                                                 self._t(v, g.face_shape(1), "v"),
                                                 self._t(w, g.face_shape(2), "w"), ct.byref(m)),
                   "paris_max_divergence")
        return m.value


class Batch:
    """Many independent projections of uneven grid sizes in one persistent
    launch (paris_batch_*).  Arrays are pooled: one device buffer per kind
    (C, p: cells; u, v, w: faces), instances concatenated in order."""

    def __init__(self, grids, opts: _abi.Opts | None = None, device=None, stream=None, **kw):
        self.lib = _abi.load()
        self.grids = [Grid(g.nx, g.ny, g.nz, g.h, tuple(g.bc)) for g in grids]
        self.n = len(self.grids)
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else
                                   torch.device(device).index or 0)
        with torch.cuda.device(self.device):
            self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.opts = opts if opts is not None else default_opts(**kw)
        arr = (_abi.Grid * self.n)(*[_grid_struct(g) for g in self.grids])
        self._ptr = ct.c_void_p()
        with torch.cuda.device(self.device):
            _abi.check(self.lib.paris_batch_create(ct.byref(self._ptr), self.n, arr, ct.byref(self.opts),
                                                   ct.c_void_p(self.stream.cuda_stream)),
                       "paris_batch_create")
        offs = [(ct.c_int64 * (self.n + 1))() for _ in range(4)]
        _abi.check(self.lib.paris_batch_layout(self._ptr, *offs), "paris_batch_layout")
        self.offsets = {k: np.array(o[:], dtype=np.int64) for k, o in zip(("cells", "u", "v", "w"), offs)}

    def close(self):
        if getattr(self, "_ptr", None) and self._ptr.value:
            self.lib.paris_batch_destroy(self._ptr)
            self._ptr = ct.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @property
    def launch_ctas(self):
        return int(self.lib.paris_batch_launch_ctas(self._ptr))

    def pack(self, arrays, kind):
        """Concatenate per-instance numpy/torch arrays of one kind into a device pool."""
        off = self.offsets["cells" if kind in ("C", "p") else kind]
        pool = torch.empty(int(off[-1]), dtype=torch.float64, device=self.device)
        for i, a in enumerate(arrays):
            t = a if isinstance(a, torch.Tensor) else torch.from_numpy(np.ascontiguousarray(a))
            pool[off[i]:off[i + 1]] = t.reshape(-1).to(self.device, torch.float64)
        return pool

    def unpack(self, pool, kind):
        """Views of a pool as per-instance arrays (numpy shape conventions)."""
        off = self.offsets["cells" if kind in ("C", "p") else kind]
        out = []
        for i, g in enumerate(self.grids):
            shape = g.shape if kind in ("C", "p") else g.face_shape("uvw".index(kind))
            out.append(pool[off[i]:off[i + 1]].view(shape))
        return out

    def _check_pool(self, x, kind):
        off = self.offsets["cells" if kind in ("C", "p") else kind]
        if (not isinstance(x, torch.Tensor) or x.dtype != torch.float64 or not x.is_contiguous()
                or x.device != self.device or x.numel() != int(off[-1])):
            raise ValueError(f"{kind}: need a contiguous float64 pool of {int(off[-1])} on {self.device}")
        return ct.c_void_p(x.data_ptr())

    def projection_step(self, C, rho1, rho2, dt, u, v, w, p, check=True):
        """One step of every instance; u, v, w, p pools updated in place.
        rho1, rho2, dt: sequences of n values.  Returns a list of stats dicts."""
        st = (_abi.Stats * self.n)()
        arr = lambda x: (ct.c_double * self.n)(*[float(a) for a in x])
        s = self.lib.paris_batch_projection_step(self._ptr, self._check_pool(C, "C"), arr(rho1), arr(rho2),
                                                 arr(dt), self._check_pool(u, "u"), self._check_pool(v, "v"),
                                                 self._check_pool(w, "w"), self._check_pool(p, "p"), st)
        stats = [x.as_dict() for x in st]
        if check:
            _abi.check(s, "paris_batch_projection_step", stats)
        return stats

    def autotune(self, C, rho1, rho2, dt, u, v, w, cache_path=None):
        """Pick sweeps, omega and CTAs per SM by timing; returns the best time (ms)."""
        arr = lambda x: (ct.c_double * self.n)(*[float(a) for a in x])
        best = ct.c_double(0.0)
        _abi.check(self.lib.paris_batch_autotune(
            self._ptr, self._check_pool(C, "C"), arr(rho1), arr(rho2), arr(dt), self._check_pool(u, "u"),
            self._check_pool(v, "v"), self._check_pool(w, "w"),
            cache_path.encode() if cache_path else None, ct.byref(best)), "paris_batch_autotune")
        return best.value

    def tuning(self):
        nu, om, bps = ct.c_int(), ct.c_double(), ct.c_int()
        _abi.check(self.lib.paris_batch_get_tuning(self._ptr, ct.byref(nu), ct.byref(om), ct.byref(bps)),
                   "paris_batch_get_tuning")
        return nu.value, om.value, bps.value
