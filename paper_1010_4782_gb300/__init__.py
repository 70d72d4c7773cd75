"""GB300-native staggered-fermion even-odd CG (sm_103a CUDA kernels behind a C ABI).

The CUDA library is loaded on first use of the binding; there is no CPU
fallback.
"""
__version__ = "0.1.0"
