"""FP64 CPU oracle for the continuous quadratic knapsack problem (CQK).

TEST INFRASTRUCTURE -- not part of the product path.  Only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py``'s cpu_baseline / reference arm may
import it.  It shares no code with the CUDA library in ``paper_2603_15910_b300``
and never imports it; the only code both sides use is the seeded input
generator module ``paper_2603_15910_b300.workloads`` (random arrays, none of the
method's arithmetic).

Problem (Sec. 1, eq. (CQK)):  min 1/2 x'Dx - a'x  s.t.  b'x = r,  l <= x <= u,
with D = diag(d), d > 0, b > 0; bounds may be infinite.

Parts:
  ``reference``  ctypes wrappers of ``cqk_oracle.c``: the paper's sequential
                 algorithms (Alg. 1-4, eq. (CQKlambda0)) and the exact
                 sort-based solvers.
  ``exact``      numpy: brute-force active-set enumeration, KKT residuals, the
                 l1-ball projection by Lemma 3.2, and the implicit-function
                 gradient of the solution map.

Parity status: every routine here is pinned by a ``-m "not gpu"`` test against
something other than itself (brute force, closed forms, a second algorithm,
finite differences); see tests/test_oracle_*.py.
"""
from .reference import (  # noqa: F401
    EPS34_F64,
    EPS34_F32,
    STOP_NAMES,
    x_of_lambda,
    phi,
    lambda0_formula,
    lambda0_warm,
    breakpoint_search,
    newton_cqk,
    solve_sort,
    condat_init,
    condat_chunks,
    condat_chunks_warm,
    condat_project,
    newton_simplex,
    project_simplex_sort,
)
from .exact import (  # noqa: F401
    brute_force_cqk,
    kkt_residuals,
    project_simplex,
    project_l1,
    grad_cqk,
    grad_simplex,
    grad_l1,
    lambda0_simplex_formula,
)
