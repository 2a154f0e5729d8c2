"""Seeded synthetic inputs shared by the oracle tests, the CUDA tests and bench.py.

This package builds gate lists and workload descriptions only. It holds none of
the tableau arithmetic: no gate rule, rowsum, phase or measurement logic lives
here, so neither side of a parity test can borrow the other's mathematics
through it.
"""

from .circuits import *  # noqa: F401,F403
