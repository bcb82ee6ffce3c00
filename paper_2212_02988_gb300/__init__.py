"""GB300 (sm_103a) implementation of the PRISM filter hot path (arXiv 2212.02988).

The compute path is libprism.so (CUDA kernels behind the C ABI of
include/prism.h); this package is its thin Python binding.
"""
from .filter import Filter, PrismError, config, make_state, normal_equations_noalloc, state_arrays

__all__ = ["Filter", "PrismError", "config", "make_state", "normal_equations_noalloc", "state_arrays"]
