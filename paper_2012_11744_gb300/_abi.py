"""ctypes declarations of the C ABI in include/paris.h (argument marshalling only).

The shared library is built in-tree by ``build.py``; loading fails loudly
when it is missing: there is no CPU fallback for any entry point.
"""
from __future__ import annotations

import ctypes as ct
import os
import threading

from . import build as _build

PARIS_OK = 0
PARIS_ERR_INVALID_ARG = 1
PARIS_ERR_CUDA = 2
PARIS_ERR_NOT_CONVERGED = 3
PARIS_ERR_NONFINITE = 4
PARIS_ERR_TIMEOUT = 5
PARIS_ERR_NO_MEMORY = 6

PERIODIC = 0
WALL = 1
FP64 = 0
MIXED = 1
SMOOTH_RBGS = 0
SMOOTH_JACOBI = 1
SMOOTH_RBGS_2PASS = 2


class Grid(ct.Structure):
    _fields_ = [("nx", ct.c_int), ("ny", ct.c_int), ("nz", ct.c_int), ("h", ct.c_double),
                ("bc", ct.c_int * 3)]


class Opts(ct.Structure):
    _fields_ = [("tol", ct.c_double), ("max_iter", ct.c_int), ("precision", ct.c_int),
                ("nu1", ct.c_int), ("nu2", ct.c_int), ("omega", ct.c_double),
                ("smoother", ct.c_int), ("coarse_max_cells", ct.c_int),
                ("inner_tol", ct.c_double), ("fallback", ct.c_int), ("slab_planes", ct.c_int),
                ("half_coefficients", ct.c_int), ("level0_density", ct.c_int),
                ("level0_tiles", ct.c_int), ("level0_half_rho", ct.c_int),
                ("coarse_tail", ct.c_int)]


class KernelProf(ct.Structure):
    _fields_ = [("launches", ct.c_int64), ("timed", ct.c_int64), ("ms", ct.c_double),
                ("bytes", ct.c_double)]


K_SMOOTH0, K_RESTRICT0, K_PROLONG0, K_MATVEC0, K_RESID64 = range(5)
K_NAMES = ("smooth0", "restrict0", "prolong0", "matvec0", "resid64", "coarse", "field", "setup", "krylov",
           "project")
# classes of single kernels with an algorithmic byte count (the others group many launches)
K_BYTES = ("smooth0", "restrict0", "prolong0", "matvec0", "resid64")


class Stats(ct.Structure):
    _fields_ = [("iters", ct.c_int), ("outer_iters", ct.c_int), ("rel_res_l2", ct.c_double),
                ("rel_res_linf", ct.c_double), ("mean_b_removed", ct.c_double),
                ("fell_back", ct.c_int), ("converged", ct.c_int), ("levels", ct.c_int)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_P = ct.c_void_p
_D = ct.c_double
_lib = None
_lock = threading.Lock()

# name -> (restype, argtypes); every function declared in include/paris.h
SIGNATURES = {
    "paris_default_opts": (None, [ct.POINTER(Opts)]),
    "paris_create": (ct.c_int, [ct.POINTER(_P), ct.POINTER(Grid), ct.POINTER(Opts), _P]),
    "paris_destroy": (ct.c_int, [_P]),
    "paris_set_opts": (ct.c_int, [_P, ct.POINTER(Opts)]),
    "paris_face_coeffs": (ct.c_int, [_P, _P, _D, _D, _P, _P, _P]),
    "paris_divergence": (ct.c_int, [_P, _P, _P, _P, _D, _P, ct.POINTER(_D)]),
    "paris_divergence_noalloc": (ct.c_int, [ct.POINTER(Grid), _P, _P, _P, _D, _P, _P, _P]),
    "paris_poisson_solve": (ct.c_int, [_P, _P, _P, _P, _P, _P, ct.POINTER(Stats)]),
    "paris_project": (ct.c_int, [_P, _P, _P, _P, _P, _D, _P, _P, _P]),
    "paris_projection_step": (ct.c_int, [_P, _P, _D, _D, _D, _P, _P, _P, _P, ct.POINTER(Stats)]),
    "paris_projection_step_host": (ct.c_int, [_P, _P, _D, _D, _D, _P, _P, _P, _P,
                                              ct.POINTER(Stats)]),
    "paris_project_adjoint": (ct.c_int, [_P, _P, _P, _P, _P, _D, _P, _P, _P, _P, _P, _P, _P, _P,
                                         _P, _P, ct.POINTER(Stats)]),
    "paris_face_coeffs_adjoint": (ct.c_int, [_P, _D, _D, _P, _P, _P, _P, _P, _P, _P]),
    "paris_predictor_forcing": (ct.c_int, [_P, _P, _P, _D, _D, _D, _D, _D, _D, _D, _P, _P, _P, _P, _P, _P]),
    "paris_projection_step_forced": (ct.c_int, [_P, _P, _P, _D, _D, _D, _D, _D, _D, _D, _P, _P, _P, _P,
                                                ct.POINTER(Stats)]),
    "paris_set_solid": (ct.c_int, [_P, _P]),
    "paris_marker_function": (ct.c_int, [_P, _P, _P, _P, _D, _P, ct.POINTER(Stats)]),
    "paris_free_surface_step": (ct.c_int, [_P, _P, _D, _D, _P, _P, _P, _P, _D, _P, _P, _P, _P, _P,
                                           ct.POINTER(Stats)]),
    "paris_phantom_projection": (ct.c_int, [_P, _P, _P, _P, _P, _P, ct.POINTER(Stats)]),
    "paris_face_viscosity": (ct.c_int, [_P, ct.c_int, _P, _D, _D, _D, _D, _P]),
    "paris_viscous_solve": (ct.c_int, [_P, ct.c_int, _P, _D, _P, _P, _D, ct.c_int, ct.POINTER(Stats)]),
    "paris_viscous_solve_mg": (ct.c_int, [_P, ct.c_int, _P, _D, _P, _P, _D, ct.c_int, ct.POINTER(Stats)]),
    "paris_batch_create": (ct.c_int, [ct.POINTER(_P), ct.c_int, ct.POINTER(Grid), ct.POINTER(Opts), _P]),
    "paris_batch_destroy": (ct.c_int, [_P]),
    "paris_batch_layout": (ct.c_int, [_P, ct.POINTER(ct.c_int64), ct.POINTER(ct.c_int64),
                                      ct.POINTER(ct.c_int64), ct.POINTER(ct.c_int64)]),
    "paris_batch_launch_ctas": (ct.c_int, [_P]),
    "paris_batch_projection_step": (ct.c_int, [_P, _P, ct.POINTER(_D), ct.POINTER(_D), ct.POINTER(_D),
                                               _P, _P, _P, _P, ct.POINTER(Stats)]),
    "paris_batch_autotune": (ct.c_int, [_P, _P, ct.POINTER(_D), ct.POINTER(_D), ct.POINTER(_D), _P, _P,
                                        _P, ct.c_char_p, ct.POINTER(_D)]),
    "paris_batch_get_tuning": (ct.c_int, [_P, ct.POINTER(ct.c_int), ct.POINTER(_D),
                                          ct.POINTER(ct.c_int)]),
    "paris_residual_norms": (ct.c_int, [_P, _P, _P, _P, _P, _P, ct.POINTER(_D), ct.POINTER(_D)]),
    "paris_max_divergence": (ct.c_int, [_P, _P, _P, _P, ct.POINTER(_D)]),
    "paris_check_arithmetic": (ct.c_int, [_P, ct.c_int64, ct.c_int, ct.POINTER(ct.c_int64), _P]),
    "paris_stream_rates": (ct.c_int, [_P, _P, _P, _P, ct.c_int64, ct.c_int, ct.POINTER(ct.c_double),
                                      ct.POINTER(ct.c_double), _P]),
    "paris_profile": (ct.c_int, [_P, ct.c_int]),
    "paris_profile_read": (ct.c_int, [_P, ct.c_int, ct.POINTER(KernelProf)]),
    "paris_launch_count": (ct.c_int64, []),
    "paris_face_count": (ct.c_int64, [_P, ct.c_int]),
    "paris_cell_count": (ct.c_int64, [_P]),
    "paris_status_string": (ct.c_char_p, [ct.c_int]),
    "paris_last_cuda_error": (ct.c_char_p, []),
}


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libparis.so (building it first when it is missing or stale and
    nvcc is available).  Raises if the library cannot be loaded."""
    global _lib
    with _lock:
        if _lib is None:
            if build_if_missing and _build.needs_build():
                _build.build()
            if not os.path.exists(_build.LIB):
                raise RuntimeError("libparis.so is not built; run paper_2012_11744_gb300/build.py")
            lib = ct.CDLL(_build.LIB)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


class ParisError(RuntimeError):
    def __init__(self, status: int, where: str, stats=None):
        self.status = status
        self.stats = stats
        lib = load()
        msg = lib.paris_status_string(status).decode()
        if status == PARIS_ERR_CUDA:
            msg += " [" + lib.paris_last_cuda_error().decode() + "]"
        super().__init__(f"{where}: {msg} (status {status})")


def check(status: int, where: str, stats=None):
    if status != PARIS_OK:
        raise ParisError(status, where, stats)
