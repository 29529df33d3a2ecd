"""GB300-native solver for the mixed-quadrature Shakhov lattice Boltzmann model
of Couette flow (arXiv:1702.01335).

The solver is the C ABI of include/lbs.h, implemented by the CUDA kernels in
csrc/ and built in-tree into _build/liblbs.so; `lbs` is its Python binding.
"""
from .lbs import (LBS_ERR_ARG, LBS_ERR_NO_CONVERGENCE, LBS_ERR_NONFINITE, LBS_ERR_TIMEOUT, LBS_FP32,  # noqa: F401
                  LBS_FP64, MOMENT_NAMES, PROFILE_NAMES, VISC_POWER, VISC_SUTHERLAND, Instance, LbsError,
                  Solver, State, load, quadrature)
