"""GB300 (sm_103a) implicit one-sided Hari-Zimmermann GHSVD solver.

The compute path is the CUDA library ``libghsvd.so`` (C ABI in
include/ghsvd.h); ``ghsvd`` is its Python binding.
"""
from . import ghsvd  # noqa: F401
from .ghsvd import Solver  # noqa: F401
