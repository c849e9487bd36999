"""GB300 (sm_103a) Magnus-Chebyshev Floquet propagator (arXiv:1508.07621).

The compute path is libfloquet.so (C ABI declared in include/floquet.h, CUDA kernels in
csrc/); this package is its ctypes binding plus small conveniences that allocate device
memory through torch.  Importing it fails if the library has not been built.
"""
from ._binding import *  # noqa: F401,F403
from .api import (Plan, fidelity_loss, floquet_analysis, floquet_states, overlap_phase_error,  # noqa: F401
                  unitarity_defect, workspace)
