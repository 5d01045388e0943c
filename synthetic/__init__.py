"""Seeded synthetic inputs shared by the oracle-side tests and the CUDA path.

This package only draws models, acquisition geometry and the source wavelet.
It holds none of the method's arithmetic (no wave equation, no gradient, no
Lame conversion), so both sides can use it without sharing computation.
"""
from .workloads import (  # noqa: F401
    Workload,
    ricker,
    config0,
    config1,
    config2,
    config3,
    config4,
    tiny_borehole,
    homogeneous,
    PRESETS,
)
