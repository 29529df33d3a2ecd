"""GB300-native solver for the mixed-quadrature Shakhov lattice Boltzmann model
of Couette flow (arXiv:1702.01335).

The solver is the C ABI of include/lbs.h, implemented by the CUDA kernels in
csrc/ and built in-tree into _build/liblbs.so; `lbs` is its Python binding.
"""
from .lbs import (LBS_FP32, LBS_FP64, MOMENT_NAMES, PROFILE_NAMES, VISC_POWER,  # noqa: F401
                  VISC_SUTHERLAND, Instance, LbsError, Solver, load, quadrature)
