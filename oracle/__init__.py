"""CPU oracle of the BSDE solver (Labart & Lelong, Algorithm 2) in FP64.

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and the
cpu_baseline leg of bench.py, never by the product package.  It shares no code
with the CUDA library.  Every function is pinned by a `-m "not gpu"` test in
tests/test_oracle_*.py against values fixed by the paper or by mathematics
(closed forms, invariants, library routines, known-answer vectors).
"""
from . import bsde_oracle, closed_forms  # noqa: F401
