"""GB300 (sm_103a) multigrid pressure Poisson solver: -div((1/rho) grad p) = b.

The compute path is the CUDA library ``lib/libmgpoisson.so`` (C ABI in
``include/mg.h``); this package is its Python binding.  ``_lib`` holds the
ctypes marshalling with the C names, ``solver`` a Solver object and the
``PoissonSolve`` (from face coefficients) and ``PoissonSolveFractions`` (from
phase fractions) autograd Functions.  Importing the package does not load the
library; the first call does, and fails loudly if it was not built.
"""
from . import _lib
from ._lib import (MG_ERR_ARG, MG_ERR_CUDA, MG_ERR_DENSITY, MG_ERR_DIVERGED, MG_ERR_NOT_CONVERGED,
                   MG_ERR_OOM, MG_ERR_STATE, MG_F32, MG_F64, MG_FP64, MG_MIXED, MG_OK,
                   MG_PROLONG_CONSTANT, MG_PROLONG_TRILINEAR)
from .solver import MgError, PoissonSolve, PoissonSolveFractions, Solver

__all__ = ["Solver", "PoissonSolve", "PoissonSolveFractions", "MgError", "_lib"]
