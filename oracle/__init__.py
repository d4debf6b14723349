"""FP64 CPU oracle for the HISQ multi-rhs Dslash and CG (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline legs of
``bench.py`` may import this package. The CUDA library never does.
"""
from .hisq_oracle import *  # noqa: F401,F403
from . import hisq_oracle  # noqa: F401
