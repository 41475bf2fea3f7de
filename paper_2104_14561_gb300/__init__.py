"""GB300 (sm_103a) Feynman-Kac exit-probability march (arXiv 2104.14561).

The compute path is libfk_gb300.so (CUDA kernels behind the C ABI of
include/fk.h); this package only marshals PyTorch tensors into it.
"""
from .fk import (ExitProbability, Plan, PlanSpec, exit_probability, gauss_hermite,  # noqa: F401
                 measure_fma_rate, runaway_quench_params, solve_batched)
from ._lib import FkError, load  # noqa: F401
