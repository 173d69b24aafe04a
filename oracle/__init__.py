"""CPU oracle for the MCQSG hot path (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` import this package.  The product library never does.  The
oracle is plain C (``qisg_oracle.c``) driven through ctypes, one int8 spin per
(sample, replica, walker, site), and shares no code with the CUDA path.
"""
from .oracle import *  # noqa: F401,F403
