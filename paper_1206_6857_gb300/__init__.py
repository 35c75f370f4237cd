"""GB300-native epsilon-relative Gaussian summation (Lee & Gray, "Faster
Gaussian Summation: Theory and Experiment").

The computation lives in the CUDA library built from csrc/ (C ABI in
include/gs.h); gs.py is its thin ctypes binding.
"""
from . import build  # noqa: F401
