"""FP64 CPU oracle for the staggered-grid Stokes smoothers (test infrastructure only).

Only the tests, the smoke check and the benchmark's CPU-baseline leg may import
this package.  It shares no code with the CUDA library.
"""
from .oracle import *  # noqa: F401,F403
from . import oracle3d  # noqa: F401  (the 3D oracle)
