"""GB300-native ordered greedy code sweep (Paliwal et al., "Generating Binary
Optimal Codes Using Heterogeneous Parallel Computing").

The compute lives in ``libgc.so`` (CUDA kernels for sm_103a behind the C ABI
declared in ``include/gc.h``); :mod:`paper_1507_05398_gb300.gc` is a thin
ctypes binding with the same names.  PyTorch is used only for device memory
and streams.
"""
from .gc import *  # noqa: F401,F403
from .gc import __all__  # noqa: F401
