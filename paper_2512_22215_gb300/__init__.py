"""GB300 LDU pressure solve: laplacian assembly, Amul, DIC/diagonal PCG,
mixed-precision refinement, adjoint and batched solves, as sm_103a CUDA
kernels behind a C ABI (include/spuma.h)."""
from ._lib import (F32, F64, MIXED, MIXED_RESTART, PRECOND_DIAGONAL, PRECOND_DIC, PRECOND_DILU, PRECOND_NONE, Controls, Perf,
                   SpumaError, lib)
from .core import LduMesh, SolverControls, BatchSolve, GamgSolver, solve_host
from .autograd import LaplacianAssembly, PressureSolve, assemble_laplacian, pressure_solve

__all__ = ["LduMesh", "SolverControls", "BatchSolve", "GamgSolver", "PressureSolve", "pressure_solve", "LaplacianAssembly",
           "assemble_laplacian", "solve_host",
           "Controls", "Perf", "SpumaError", "lib", "F64", "F32", "MIXED", "MIXED_RESTART", "PRECOND_NONE",
           "PRECOND_DIAGONAL", "PRECOND_DIC", "PRECOND_DILU"]
