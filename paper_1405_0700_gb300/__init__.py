"""GB300 (sm_103a) implementation of the Wilson-Dirac hopping operator and its
Krylov solvers, after "PLQCD library for Lattice QCD on multi-core machines".

The compute path is ``libplq.so`` (CUDA kernels behind the C ABI in
``include/plq.h``); ``paper_1405_0700_gb300.plq`` is its ctypes binding.
"""
from .plq import (  # noqa: F401
    DF64,
    F16,
    F32,
    F64,
    MAX_RHS,
    Context,
    PLQError,
    SolveInfo,
    SolverParams,
    lib,
)
