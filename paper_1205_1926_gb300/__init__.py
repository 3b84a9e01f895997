"""GB300-native TFETI solver for one-time-step von Mises elastoplasticity.

The compute path is the in-tree CUDA library ``_lib/libtfeti_gb300.so`` (C ABI
in ``include/tfeti.h``); this package only builds and binds it.
"""
from .binding import (Context, Plan, TfetiError, load, library_path, make_problem, PRECOND_LUMPED,  # noqa: F401
                      PRECOND_NONE, PRECOND_DIRICHLET, SIGNATURES, time_step_cases, measure_fp64_fma,
                      COARSE_AUTO, COARSE_DENSE, COARSE_PLANES)
