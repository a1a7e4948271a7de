"""Serial FP64 CPU oracle of the aggregation-AMG Krylov method (arXiv 2007.00056).

TEST INFRASTRUCTURE ONLY: imported by the test suite, by ``__graft_entry__.smoke``
and by the CPU-baseline leg of ``bench.py``.  The CUDA library never uses it.

The arithmetic lives in ``amg_oracle.c`` (plain C, built with
``-O2 -ffp-contract=off``).  This module compiles it on first use and wraps it
with ctypes and numpy arrays.
"""
from .oracle import (  # noqa: F401
    build,
    lib,
    Params,
    Hierarchy,
    spmv,
    check_csr,
    match_greedy,
    match_rounds,
    nhem,
    aggregates,
    galerkin,
    dense_solve,
    OK,
    ERR_INVALID_ARG,
    ERR_INVALID_CSR,
    ERR_ZERO_DIAG,
    ERR_OOM,
    ERR_BREAKDOWN,
    ERR_NOT_CONVERGED,
)
