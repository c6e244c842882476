"""CPU oracle for multinomial resampling (test infrastructure only).

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA library
in ``paper_2604_01356_gb300``.
"""
from .oracle import *  # noqa: F401,F403
