"""CPU FP64 oracle of the AMG-DD solve phase (test infrastructure only).

Only the tests, the smoke check and the CPU-baseline leg of the benchmark use
this package. The product library never imports it.
"""
from .oracle import Oracle, build_oracle, kappa_gradient, oracle_lib, set_threads  # noqa: F401
