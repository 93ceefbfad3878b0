"""FP64 CPU oracle for LS-AMG-DD (test infrastructure only).

This package is the slow, plain reference that the CUDA path is checked
against.  Only the test-suite, ``__graft_entry__.smoke()`` and ``bench.py``'s
CPU-baseline / reference leg may import it; the library path never does.
It shares no code with the CUDA library: the only common dependency is the
seeded input generator ``fegen``.
"""
from .lsamg_oracle import *  # noqa: F401,F403
