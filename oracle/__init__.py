"""CPU FP64 oracle for the upwind Eikonal discretisation (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA solver.
"""
from .oracle import (  # noqa: F401
    SOURCE,
    Oracle,
    OracleError,
    apply_T,
    build,
    cells,
    default,
    fmm,
    fmsm,
    fsm,
    jacobi,
    lsm,
    node_update,
)
