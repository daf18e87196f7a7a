"""GB300-native preconditioned steepest descent (PSD) for the periodic
finite-difference regularized p-Laplacian problems of Feng, Salgado, Wang &
Wise (arXiv:1607.01475).

The compute path is the CUDA library ``libpsd.so`` (C ABI in
``include/psd.h``); this package only marshals arguments to it.  There is no
CPU fallback: if the library cannot be loaded, every call raises.
"""

from ._lib import (  # noqa: F401
    PSD_FP64, PSD_MIXED, Batch, PSDError, Solver, lib_path, load_library,
    psd_create, psd_destroy, psd_precond_solve, psd_residual, psd_residual_f32,
    psd_residual_noalloc, psd_hvp, psd_adjoint,
    psd_solve, psd_status_string,
)
