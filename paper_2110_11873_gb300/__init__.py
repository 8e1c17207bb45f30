"""GB300-native matrix-free transfer operator and Krylov solvers for the 1D
two-level-atom CRD polarized transfer problem (Benedusi et al. 2021).

The compute path is the C-ABI library librtkrylov.so (include/rt_krylov.h);
this package only marshals arguments to it.
"""
from . import _native
from .api import Problem, Server, SolveResult, TorchAllocator

__all__ = ["Problem", "Server", "SolveResult", "TorchAllocator", "_native"]
