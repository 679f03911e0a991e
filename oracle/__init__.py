"""FP64 CPU oracle of GS-SLAM's differentiable RGB-D splatting (test infrastructure).

This package is test infrastructure.  Only `tests/`, `__graft_entry__.smoke()`
and the CPU-baseline leg of `bench.py` may import it.  The CUDA path never
imports it and it imports nothing from the CUDA path; the two share no code.

Parity status: every function here is pinned by the `-m "not gpu"` tests in
`tests/test_oracle_*.py` (closed forms, the supplement's derivative formulas,
library special cases, brute force and central finite differences).
"""
from .gs_oracle import *  # noqa: F401,F403
