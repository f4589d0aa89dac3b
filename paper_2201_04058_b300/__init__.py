"""B300-native metapath-query engine (hot path of the ATRAPOS method, arXiv 2201.04058).

The compute path is the CUDA library ``_lib/libmp.so`` behind the C ABI of
``include/mp.h``; ``paper_2201_04058_b300.mp`` is a thin ctypes binding with the same
names. There is no CPU fallback: importing the binding fails if the library is missing.
"""
from .mp import *  # noqa: F401,F403
