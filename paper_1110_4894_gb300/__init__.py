"""GB300 (sm_103a) 3D ray-bundle gravitational lensing.

A thin ctypes binding over ``librt3d.so`` (C ABI in include/rt3d.h).  Every
step of the computation runs in the library's CUDA kernels; this module only
marshals numpy arrays and device pointers.  There is no CPU fallback: if the
library cannot be loaded, every entry point raises.
"""
from ._binding import (  # noqa: F401
    CHRISTOFFEL_DERIVED, CHRISTOFFEL_PAPER, FP64, F_NEGPARITY, F_NOCROSS, F_NONFINITE, MIXED,
    SCHED_ASINH, SCHED_UNIFORM, Rt3dError, Context, histogram_combine, lib, library_path,
)
