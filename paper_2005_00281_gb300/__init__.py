"""GB300-native hot path of borehole acoustic full-waveform inversion.

The compute runs in libbh (CUDA, sm_103a) behind the C ABI of include/bh.h;
this package holds the build step and a thin ctypes binding.
"""
from .build import build_library, LIB  # noqa: F401
