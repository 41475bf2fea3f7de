"""GB300 (sm_103a) Feynman-Kac exit-probability march (arXiv 2104.14561).

The compute path is libfk_gb300.so (CUDA kernels behind the C ABI of
include/fk.h); this package only marshals PyTorch tensors into it.
"""
from .fk import Plan, PlanSpec, gauss_hermite, solve_batched  # noqa: F401
from ._lib import FkError, load  # noqa: F401
