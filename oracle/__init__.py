"""FP64 CPU oracle for the PTHR hot path -- test infrastructure only.

Used by the tests, by ``__graft_entry__.smoke()`` and by the CPU baseline leg
of ``bench.py``; never by the product path.  See ``pthr_oracle.c``.
"""
from .oracle import *  # noqa: F401,F403
from .oracle import build, lib, OracleSample, run_samples_threaded  # noqa: F401
