"""GB300-native TT-rounding and TT orthogonalization (Coulaud, Giraud &
Iannacito, "On some orthogonalization schemes in Tensor Train format").

The compute path is the CUDA library ``libttgb.so`` (C ABI in
``include/ttgb.h``); ``ttgb`` is its ctypes binding.
"""
from . import build  # noqa: F401
