"""GB300 (sm_103a) smoothers for the 2D variable-viscosity Stokes velocity operator.

The compute path lives in the CUDA library ``libstokes.so`` (C ABI declared in
``include/stokes.h``); ``paper_2509_19061_gb300.api`` is its thin Python binding.
Importing the package does not load the library; the first call does, and it
raises if the library has not been built.
"""
__all__ = ["api", "inputs"]
