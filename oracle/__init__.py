"""Sequential C++ oracle of the LD-Leiden batch update (test infrastructure only).

Only the tests, the smoke check and the benchmark's CPU-baseline leg import
this package.  The library's product path never does.
"""
from .oracle import Oracle, build_oracle, decouple, PARAM_DEFAULTS  # noqa: F401
