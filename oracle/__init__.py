"""CPU oracle of the four-equation MPMC right-hand side (test infrastructure).

Only the tests, the smoke check and the benchmark's CPU-baseline leg import
this package.  The product library never does.
"""
from .oracle import Oracle, build, lib_path  # noqa: F401
