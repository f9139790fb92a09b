"""CPU oracle for warm-start APSP (test infrastructure only).

Only the tests, the package smoke check and the benchmark's CPU-baseline /
reference leg import this package.  It shares no code with the CUDA path.
"""
from . import apsp  # noqa: F401
