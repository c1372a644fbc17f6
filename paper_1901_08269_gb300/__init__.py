"""GB300-native fourth-order compact Poisson solver with immersed bodies.

The compute path is the CUDA library ``libcfp.so`` (C ABI in
``include/cfp.h``); ``paper_1901_08269_gb300.cfp`` is its thin Python binding.
Importing this package does not load the library; the binding does, and it
raises if the library is missing.
"""
__all__ = ["workloads"]
