"""FP64 CPU oracle for the dense P0 single-layer BEM capacity computation.

TEST INFRASTRUCTURE ONLY: imported by the tests, by ``__graft_entry__.smoke()``
and by the benchmark's CPU-baseline leg.  The product path never imports it.
It shares no code with the CUDA library (``paper_1901_08393_gb300``).
"""
from .oracle import *  # noqa: F401,F403
