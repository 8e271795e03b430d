"""GB300-native four-component LR-CCSD polarizabilities with FNS++ truncation.

The compute path is the CUDA library ``_lrcc.so`` (sources in ``csrc/``,
C ABI in ``include/lrcc.h``); ``lrcc`` is its ctypes binding and ``build``
compiles it for sm_103a.
"""
from .lrcc import *  # noqa: F401,F403
from .lrcc import ResidualFn, library  # noqa: F401
