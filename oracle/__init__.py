"""FP64 CPU oracle for the Feynman-Kac exit-probability march (arXiv 2104.14561).

Test infrastructure only: the test suite, the smoke check and the benchmark's
CPU-baseline leg may use it; the product path never does.
"""
from .fk_oracle import *  # noqa: F401,F403
