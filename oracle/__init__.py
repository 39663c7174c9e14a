"""CPU FP64 oracle of the QPAT reconstruction hot path -- test infrastructure.

Only `tests/`, `__graft_entry__.smoke()` and the CPU-baseline / reference leg of
`bench.py` may import this package.  It shares no code with the CUDA path:
assembled sparse matrices, exact sparse LU solves and plain loops, each step
written from the paper's equations.
"""
from .qpat_oracle import *  # noqa: F401,F403
