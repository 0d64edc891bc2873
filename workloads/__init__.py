"""Seeded synthetic inputs for the sorted-recycling solve.

This module only draws random inputs (coefficient fields, parameter
vectors, right-hand sides, arrival times).  It holds none of the solver's
arithmetic: discretisation, sorting and the Krylov solves live in the CUDA
library and, independently, in the oracle.  Both sides consume the arrays
produced here.
"""
from .grf import grf_field
from .sequences import (
    darcy2d_sequence,
    darcy2d_circle_sequence,
    darcy3d_sequence,
    convdiff2d_sequence,
    convdiff_keys,
    helmholtz2d_sequence,
    chebyshev_poisson_sequence,
    batched_chains,
    serving_stream,
    CONFIGS,
)

__all__ = [
    "grf_field",
    "darcy2d_sequence",
    "darcy2d_circle_sequence",
    "darcy3d_sequence",
    "convdiff2d_sequence",
    "convdiff_keys",
    "helmholtz2d_sequence",
    "chebyshev_poisson_sequence",
    "batched_chains",
    "serving_stream",
    "CONFIGS",
]
