"""Plain FP64 CPU oracle for the Proportional Similarity metrics.

TEST INFRASTRUCTURE ONLY: imported by the test suite, the package smoke check
and the CPU-baseline leg of the benchmark, never by the library itself.
"""
from .oracle import *  # noqa: F401,F403
