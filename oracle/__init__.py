"""Plain CPU FP64 oracle for the binned harmonic 3PCF estimator (arXiv:2408.16847).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py``; never by the library.  It shares no code with
the CUDA path.  See ``oracle.py`` for the definitions it follows.
"""
from .oracle import *  # noqa: F401,F403
from .oracle import build  # noqa: F401
