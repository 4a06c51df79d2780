"""GB300-native orbital minimization method (OMM), after Corsetti, arXiv:1312.1549.

The solver lives in the CUDA library libomm_gb300.so (C ABI: include/omm.h,
include/omm_kernels.h); this package is its thin Python binding. Importing
the package does not load the library; `OMMSolver(...)` does, and fails
loudly if the library has not been built.
"""
__all__ = ["OMMSolver", "OMMBatch", "OMMHermitian", "OMMHermitianBatch", "omm_energy"]


def __getattr__(name):
    if name in ("OMMSolver", "OMMBatch", "OMMHermitian", "OMMHermitianBatch"):
        from . import solver
        return getattr(solver, name)
    if name == "omm_energy":
        from .autograd import omm_energy
        return omm_energy
    raise AttributeError(name)
