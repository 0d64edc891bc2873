"""GB300-native sorted Krylov recycling (SKR, arXiv 2401.09516).

The computation lives in libskr.so (hand-written CUDA for sm_103a, C ABI in
include/skr.h); `paper_2401_09516_gb300._native` is its ctypes binding.
Build with `python -m paper_2401_09516_gb300.build`.
"""
from ._native import (  # noqa: F401
    Server,
    System,
    SkrError,
    convdiff2d,
    csr,
    darcy2d,
    darcy3d,
    helmholtz2d,
    poisson2d,
    skr_apply,
    skr_assemble,
    skr_last_error,
    skr_last_plan,
    skr_last_profile,
    skr_last_stats,
    skr_options_default,
    skr_poll,
    skr_release_workspace,
    skr_server_create,
    skr_server_destroy,
    skr_server_stats,
    skr_submit,
    skr_solve_sequence,
    skr_sort,
    skr_sort_grouped,
    skr_sort_noalloc,
)
