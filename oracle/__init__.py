"""Plain FP64 CPU oracle of the sharp-interface IBM fractional step.

TEST INFRASTRUCTURE ONLY: the test-suite, the smoke check and the benchmark's
CPU-baseline leg are its only users.  See oracle.py for the method map.
"""
from .oracle import build  # noqa: F401
