"""GB300 implicit-randomized-SVD PEPS contraction (libpeps) and its binding.

The compute path is the CUDA library ``libpeps.so`` (sources in ``csrc/``,
C ABI in ``include/libpeps.h``); this package only marshals arguments.
"""
from .libpeps import *  # noqa: F401,F403
