"""B300-native semismooth Newton solver for the continuous quadratic knapsack problem.

The compute path is the CUDA library ``libcqk.so`` (C ABI declared in ``include/cqk.h``,
sources in ``csrc/``); ``api`` is a thin ctypes binding over it.  Loading is lazy: importing
the package (e.g. for ``workloads``) does not need the library, but every solver call
raises ``CQKLibraryError`` if the library is missing -- there is no CPU fallback.
"""
from .api import (  # noqa: F401
    CQKLibraryError,
    Info,
    Init,
    Status,
    Workspace,
    lib_path,
    library,
    phi,
    project_l1,
    project_l1_batched,
    project_simplex,
    project_simplex_batched,
    solve,
    solve_batched,
)
