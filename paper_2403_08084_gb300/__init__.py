"""GB300-native stage-coupled implicit Runge-Kutta solver for the Q1 heat equation.

The hot path (stage operator, multigrid V-cycles, FGMRES Arnoldi reductions,
RK update, adjoint step) runs in hand-written CUDA kernels for sm_103a inside
libirk.so, behind the C ABI of include/irk.h.  Importing this package loads
that library and fails if it has not been built (there is no CPU fallback).
"""
from . import _lib
from ._lib import IRKError
from .solver import Solver
from . import tableaux
from . import adjoint

__all__ = ["Solver", "IRKError", "tableaux", "adjoint", "_lib"]
