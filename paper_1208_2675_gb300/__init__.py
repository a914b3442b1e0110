"""GB300-native Delta-matrix simulated annealing for the quadratic assignment problem.

The compute path is the C-ABI library ``libqapsa.so`` (CUDA for sm_103a, built
from ``csrc/``); ``paper_1208_2675_gb300.sa`` is a thin ctypes binding with the
same entry-point names. Importing this package loads nothing native; the
library is loaded on first use and its absence is an error, never a fallback.
"""
__all__ = ["instances"]
