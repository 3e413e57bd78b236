"""GB300-native (sm_103a) Chebyshev-accelerated subspace iteration (ChASE) on one GPU.

The compute path is the shared library libchase_gb300.so (C ABI in
include/chase_gb300.h); this package only marshals arguments to it.
"""
from .api import (Chase, ChaseEigh, colmajor, kernel_launch_count, measure_fp64_peak,  # noqa: F401
                  measure_mma_issue, set_wait_limit_ns, workspace_bytes)
from ._lib import MODES, ChaseError, load  # noqa: F401
