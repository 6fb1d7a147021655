"""GB300 (sm_103a) implementation of the PARIS one-fluid pressure projection.

The hot path -- face coefficients, divergence, multigrid-preconditioned
variable-coefficient Poisson solve, velocity correction -- runs in the CUDA
kernels of ``libparis.so`` behind the C ABI of ``include/paris.h``; this
package is the thin Python binding (argument marshalling only).
"""
from .api import (FP64, MIXED, PERIODIC, SMOOTH_JACOBI, SMOOTH_RBGS, SMOOTH_RBGS_2PASS,  # noqa: F401
                  WALL, Batch, Context, Grid, ParisError, check_arithmetic, default_opts, launch_count,
                  stream_rates)
from .autograd import projection  # noqa: F401
from .build import build  # noqa: F401

__all__ = ["projection", "Batch", "Context", "Grid", "default_opts", "ParisError", "build", "FP64", "MIXED", "PERIODIC",
           "WALL", "SMOOTH_RBGS", "SMOOTH_JACOBI", "SMOOTH_RBGS_2PASS", "launch_count", "check_arithmetic",
           "stream_rates"]
