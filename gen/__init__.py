"""Seeded synthetic inputs for the MINRES-CG solver.

This package only builds test problems (sparse matrices, eigenpairs of the
negative invariant subspace, right-hand sides).  It holds none of the solver's
arithmetic and is shared by the CPU oracle, the CUDA path's tests and the
benchmark.
"""
from .problems import (  # noqa: F401
    Problem,
    laplacian_csr,
    laplacian_smallest_eigs,
    laplacian_eigvecs,
    shift_for_negatives,
    shifted_laplacian_problem,
    random_indefinite_dense,
    dense_to_csr,
    random_sparse_symmetric,
    lap2d_64_k4,
    lap3d_128_k10,
    lap3d_128_k10_near,
    batch64_lap2d,
    shifted_lap3d_160,
    ShiftedFamily,
    shifted_family,
    small_shifted,
    small_3d,
    WORKLOADS,
)
from .saddle import saddle_96_b20x64, saddle_problem, small_saddle  # noqa: F401,E402
from .brake import BrakeSystem, brake_64, brake_system, small_brake  # noqa: F401,E402
